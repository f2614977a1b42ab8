// Warp-tile staging of low-degree neighbourhoods.
//
// A warp takes 32 consecutive vertices.  The CSR entries of the whole tile
// form one contiguous range [E0, E1); the warp streams it with coalesced
// loads, four independent loads per lane in flight, gathers one 32-bit value
// per neighbour (its PE code or cluster label) and stores (value, weight)
// pairs in shared memory.  Then every lane walks the entries of its own
// vertex there.  Compared with one sub-warp per vertex, the dependent chain
// xadj -> adjacency -> gather is paid once per tile instead of once per
// vertex, which is what bounds a per-vertex pass over a low-degree graph.
// Tiles whose range exceeds kTileE entries (a high-degree vertex inside, or a
// dense tile) are not staged: the J pass reads each lane's row straight from
// global memory, and the clustering and gain kernels let each 8-lane sub-warp
// copy the row of the vertex it serves into its quarter of the buffer.
#pragma once

#include "common.cuh"

namespace gm {

constexpr int kTileV = 32;        // vertices per warp tile
constexpr int kTileE = 512;       // staged CSR entries per warp tile
constexpr int kTileWarps = 4;     // warps per block
constexpr int kTileThreads = kTileWarps * 32;
// resident blocks per SM the tile kernels are compiled for (caps registers at
// 48 per thread: 40 warps per SM keep more gathers in flight)
constexpr int kTileMinBlocks = 10;

struct TileGraph {
  int32_t n;
  const int64_t* __restrict__ xadj;
  const int32_t* __restrict__ adj;
  const int32_t* __restrict__ adjw;
};

// Neighbourhood of one vertex: staged in shared memory or read from global.
struct StagedRow {
  const int32_t* c;
  const int32_t* w;
  __device__ __forceinline__ int32_t code(int j) const { return c[j]; }
  __device__ __forceinline__ int32_t weight(int j) const { return w[j]; }
};
template <class Gather>
struct GlobalRow {
  const int32_t* __restrict__ adj;
  const int32_t* __restrict__ adjw;
  Gather gather;
  __device__ __forceinline__ int32_t code(int j) const { return gather(adj[j]); }
  __device__ __forceinline__ int32_t weight(int j) const { return adjw[j]; }
};

// Per-lane view of its vertex after staging.
struct TileLane {
  int64_t v;      // vertex id (valid iff v < n)
  int64_t b, e;   // CSR range
  bool staged;    // entries are in shared memory at [b - E0, e - E0)
  int64_t E0;
};

// Stages the tile starting at vertex v0 (all 32 lanes call it); kTE is the
// capacity of the warp's staging arrays sc and sw.
template <int kTE = kTileE, class Gather>
__device__ __forceinline__ TileLane stage_tile(const TileGraph& g, int64_t v0, int lane, int32_t* sc, int32_t* sw,
                                               Gather gather) {
  TileLane t;
  t.v = v0 + lane;
  const bool valid = t.v < g.n;
  t.b = valid ? g.xadj[t.v] : 0;
  t.e = valid ? g.xadj[t.v + 1] : 0;
  const int last = (int)min((int64_t)31, (int64_t)g.n - 1 - v0);
  t.E0 = __shfl_sync(0xffffffffu, t.b, 0);
  const int64_t E1 = __shfl_sync(0xffffffffu, t.e, last);
  const int64_t span = E1 - t.E0;
  t.staged = span <= kTE;
  if (t.staged) {
    // every load of the tile is issued before any is used: one round trip
    // for the adjacency and weights, one for the gathers
    constexpr int kQ = kTE / 32;
    int32_t u[kQ];
#pragma unroll
    for (int q = 0; q < kQ; q++) {
      const int jj = q * 32 + lane;
      u[q] = (jj < span) ? g.adj[t.E0 + jj] : 0;
      if (jj < span) sw[jj] = g.adjw[t.E0 + jj];
    }
#pragma unroll
    for (int q = 0; q < kQ; q++) {
      const int jj = q * 32 + lane;
      if (jj < span) u[q] = gather(u[q]);
    }
#pragma unroll
    for (int q = 0; q < kQ; q++) {
      const int jj = q * 32 + lane;
      if (jj < span) sc[jj] = u[q];
    }
  }
  __syncwarp();
  return t;
}

// As stage_tile, with each staged entry one 64-bit word (value, weight) in
// scw: a scan over a staged row then costs one shared load per entry.
template <int kTE = kTileE, class Gather>
__device__ __forceinline__ TileLane stage_tile_packed(const TileGraph& g, int64_t v0, int lane, int2* scw,
                                                      Gather gather) {
  TileLane t;
  t.v = v0 + lane;
  const bool valid = t.v < g.n;
  t.b = valid ? g.xadj[t.v] : 0;
  t.e = valid ? g.xadj[t.v + 1] : 0;
  const int last = (int)min((int64_t)31, (int64_t)g.n - 1 - v0);
  t.E0 = __shfl_sync(0xffffffffu, t.b, 0);
  const int64_t E1 = __shfl_sync(0xffffffffu, t.e, last);
  const int64_t span = E1 - t.E0;
  t.staged = span <= kTE;
  if (t.staged) {
    constexpr int kQ = kTE / 32;
    int32_t u[kQ], w[kQ];
#pragma unroll
    for (int q = 0; q < kQ; q++) {
      const int jj = q * 32 + lane;
      u[q] = (jj < span) ? g.adj[t.E0 + jj] : 0;
      w[q] = (jj < span) ? g.adjw[t.E0 + jj] : 0;
    }
#pragma unroll
    for (int q = 0; q < kQ; q++) {
      const int jj = q * 32 + lane;
      if (jj < span) u[q] = gather(u[q]);
    }
#pragma unroll
    for (int q = 0; q < kQ; q++) {
      const int jj = q * 32 + lane;
      if (jj < span) scw[jj] = make_int2(u[q], w[q]);
    }
  }
  __syncwarp();
  return t;
}

// Worker of sub-warp `sub` in round r of a tile whose lanes with `work` set
// are served four at a time in lane order: the lane of rank 4 r + sub among
// the set bits (-1 if none).  `rank` is the lane's own rank among them.
__device__ __forceinline__ int tile_worker_ranked(unsigned work, int rank, int round, int sub, int lane) {
  const bool mine = ((work >> lane) & 1u) && (rank >> 2) == round;
  unsigned m = __ballot_sync(0xffffffffu, mine);
  for (int k = 0; k < sub && m; k++) m &= m - 1;
  return m ? __ffs(m) - 1 : -1;
}

// Work queue of one warp tile: the lanes with `work` set are served four at a
// time, one per 8-lane sub-warp.  For the r-th round, sub-warp s takes the
// worker of rank 4r + s.  Returns the source lane of this lane's sub-warp
// (-1 when the sub-warp has no worker this round).
__device__ __forceinline__ int tile_worker(unsigned work, int round, int sub) {
  int want = 4 * round + sub;
  unsigned m = work;
  while (m && want > 0) {
    m &= m - 1;
    want--;
  }
  return m ? __ffs(m) - 1 : -1;
}

}  // namespace gm
