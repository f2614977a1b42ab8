// Refinement engine: objective J, block weights, unconstrained label
// propagation (Alg. 4), weak / strong rebalancing (Alg. 5 and its strong
// variant, edge-cut loss) and the overall refinement driver (Alg. 6) with its
// state machine on the device.
//
// Work split by degree.  A vertex of degree <= 32 is handled by an 8-lane
// sub-warp that keeps its (up to 32) neighbour PEs and edge weights in
// registers; gains of every neighbouring PE are evaluated by shuffles, so the
// per-vertex connectivity table of Section 4.2 never leaves registers.  A
// vertex of degree 33..255 gets one warp with its own dense shared-memory
// connectivity array over the PE code space, and a larger one a whole CTA
// with one such array; per-level group sums of that array give the gain of
// every candidate PE in O(levels).
#include <atomic>
#include <chrono>
#include <type_traits>
#include <algorithm>
#include <mutex>

#include "engine.h"
#include "tile.cuh"
#include "mid.cuh"

namespace gm {

namespace {

constexpr int kThreads = 256;
constexpr int kHiThreads = 256;

struct GraphView {
  int32_t n;
  const int64_t* __restrict__ xadj;
  const int32_t* __restrict__ adj;
  const int32_t* __restrict__ adjw;
  const int32_t* __restrict__ vw;
  int32_t mid_deg;  // rows of degree in (kLowDeg, mid_deg] get one warp; larger ones the hub kernels
};

inline GraphView view(const Level& L) { return GraphView{L.n, L.xadj, L.adj, L.adjw, L.vw, L.mid_deg}; }

__host__ __device__ inline int bits_for_n(int64_t x) {  // smallest b with x <= 2^b
  int b = 0;
  while (b < 62 && (1LL << b) < x) b++;
  return b;
}

__device__ __forceinline__ bool kind_is(const RefineState* st, int mask) {
  return (mask >> st->kind) & 1;
}

// Register-array element r (r uniform across the tile; avoids local memory).
__device__ __forceinline__ int32_t pick(const int32_t (&a)[kSlots], int r) {
  int32_t x = a[0];
#pragma unroll
  for (int i = 1; i < kSlots; i++)
    if (r == i) x = a[i];
  return x;
}

template <class Tile>
__device__ __forceinline__ int64_t tile_sum64(Tile& t, int64_t v) {
#pragma unroll
  for (int o = kSubWarp / 2; o > 0; o >>= 1) v += t.shfl_xor(v, o);
  return v;
}
template <class Tile>
__device__ __forceinline__ int32_t tile_sum32(Tile& t, int32_t v) {
#pragma unroll
  for (int o = kSubWarp / 2; o > 0; o >>= 1) v += t.shfl_xor(v, o);
  return v;
}

// ---------------------------------------------------------------------------
// block weights and J
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_block_weights(int32_t n, const int32_t* __restrict__ pi,
                                                            const int32_t* __restrict__ vw, int32_t kc,
                                                            int64_t* __restrict__ W) {
  extern __shared__ int32_t hist[];
  for (int b = threadIdx.x; b < kc; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[pi[v]], vw[v]);
  __syncthreads();
  for (int b = threadIdx.x; b < kc; b += blockDim.x)
    if (hist[b]) atomicAdd((unsigned long long*)&W[b], (unsigned long long)(int64_t)hist[b]);
}

struct GatherPi {
  const int32_t* __restrict__ pi;
  __device__ __forceinline__ int32_t operator()(int32_t u) const { return pi[u]; }
};

// Persistent grid of a warp-tile kernel: one wave of resident blocks.
inline unsigned tile_grid(Ctx& c, const void* fn, int64_t n) {
  const int64_t tiles = (n + kTileV - 1) / kTileV;
  int64_t g = (tiles + kTileWarps - 1) / kTileWarps;
  const int64_t cap = (int64_t)c.num_sms * c.resident_blocks(fn, kTileThreads, 0);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// sum_j w_j D(x, c_j) over one neighbourhood
template <class Row>
__device__ __forceinline__ int64_t row_cost(const Row& r, int deg, const int32_t* sdist, int32_t x) {
  int64_t T = 0;
  for (int j = 0; j < deg; j++) T += (int64_t)r.weight(j) * dcode(sdist, x, r.code(j));
  return T;
}

struct CtlArgs {
  int64_t lmax;
  int32_t kc;
  int32_t patience, weak_max, phi_num, phi_den;
  int32_t* tk;
  int64_t* tJ;
  int64_t* tW;
  int32_t tcap;
};

// Controller attached to a J evaluation (s == nullptr: J only).
struct EvalCtl {
  RefineState* s;
  unsigned int* ctr;  // blocks finished (zero between launches)
  const int64_t* W;
  CtlArgs a;
  int phase;
  cudaGraphConditionalHandle h;
  int use_h;
};
__device__ void eval_finish(int64_t* Jacc, const EvalCtl& ec);

// True when the J evaluation closing an Alg. 6 iteration has nothing to do:
// after an LP or weak step the step itself added its exact change of J to the
// accumulator, which the previous decision had set to the old J.
__device__ __forceinline__ bool incremental_j(const RefineState* st, int phase) {
  return st && phase == 1 && (st->kind == KIND_LP || st->kind == KIND_WEAK);
}

// J contribution of the low-degree vertices (warp tiles, one lane per vertex).
// With a controller attached, the last block to finish runs the Alg. 6
// decision on the complete J (the high-degree part is added before).
__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks) k_eval_tile(GraphView g, const int32_t* __restrict__ pi, Topo topo,
                                                            int64_t* Jacc, EvalCtl ec) {
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  __shared__ int32_t sc[kTileWarps][kTileE];
  __shared__ int32_t sw[kTileWarps][kTileE];
  load_sdist(sdist, topo);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileGraph tg{g.n, g.xadj, g.adj, g.adjw};
  if (incremental_j(ec.s, ec.phase)) {
    // after an LP or weak step Jacc already holds J (old J + the exact
    // change): the blocks only arrive, and the last one runs the decision.
    // The decision rewrites the step kind that every block reads on entry,
    // so it must wait for all of them: a block scheduled late (the SMs
    // shared with other streams' kernels) would otherwise read the next
    // step's kind and stream its tiles into the accumulator.
    eval_finish(Jacc, ec);
    return;
  }
  const int64_t ntiles = ((int64_t)g.n + kTileV - 1) / kTileV;
  int64_t acc = 0;
  for (int64_t tile = (int64_t)blockIdx.x * kTileWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kTileWarps) {
    const TileLane t = stage_tile(tg, tile * kTileV, lane, sc[warp], sw[warp], GatherPi{pi});
    const int deg = (int)(t.e - t.b);
    if (t.v < g.n && deg <= kLowDeg) {
      const int32_t p = pi[t.v];
      if (t.staged) acc += row_cost(StagedRow{sc[warp] + (t.b - t.E0), sw[warp] + (t.b - t.E0)}, deg, sdist, p);
      else acc += row_cost(GlobalRow<GatherPi>{g.adj + t.b, g.adjw + t.b, GatherPi{pi}}, deg, sdist, p);
    }
    __syncwarp();
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)Jacc, (unsigned long long)acc);
  eval_finish(Jacc, ec);
}

// The high-degree kernels below come in two forms: one warp per vertex of
// degree <= kMidDeg (`_mid`, over the whole list hi[] of degree > kLowDeg,
// skipping the larger ones) and one CTA per vertex (`_high`, over the
// positions `sel` in hi[], or all of hi[] when sel is null).
__device__ __forceinline__ int32_t hi_vertex(const int32_t* hi, const int32_t* sel, int32_t j) {
  return hi[sel ? sel[j] : j];
}

// J contribution of the vertices of degree in (kLowDeg, kMidDeg], one warp per vertex.
__global__ void __launch_bounds__(kMidThreads) k_eval_mid(GraphView g, const int32_t* __restrict__ hi, int32_t n_hi,
                                                          const int32_t* __restrict__ pi, Topo topo, int64_t* Jacc,
                                                          const RefineState* st, int phase) {
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  if (incremental_j(st, phase)) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * kMidWarps + warp; i < n_hi; i += (int64_t)gridDim.x * kMidWarps) {
    const int32_t v = hi[i];
    const int64_t b = g.xadj[v], e = g.xadj[v + 1];
    if (e - b > g.mid_deg) continue;
    const int32_t p = pi[v];
    for (int64_t x = b + lane; x < e; x += 32) acc += (int64_t)g.adjw[x] * dcode(sdist, p, pi[g.adj[x]]);
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)Jacc, (unsigned long long)acc);
}

// J contribution of the vertices of degree > kMidDeg: their entries,
// flattened in huge[] order, are taken in chunks of kHubChunk by the CTAs of
// one wave (every entry's term is independent), so no CTA waits on a hub's
// whole row; each thread follows the row of its own entries.
__global__ void __launch_bounds__(kHiThreads) k_eval_high(GraphView g, HubRows hr, const int32_t* __restrict__ pi,
                                                          Topo topo, int64_t* Jacc, const RefineState* st, int phase) {
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  if (incremental_j(st, phase)) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int64_t m_hub = hr.pre[hr.n_huge];
  int64_t acc = 0;
  for (int64_t ch = blockIdx.x; ch < hr.nchunks; ch += gridDim.x) {
    const int64_t cb = ch * kHubChunk, ce = min(cb + kHubChunk, m_hub);
    int32_t r = hr.chunk[ch];
    int64_t re = hr.pre[r + 1], x0 = 0;
    int32_t p = 0;
    bool have = false;
    for (int64_t f = cb + threadIdx.x; f < ce; f += blockDim.x) {
      while (f >= re) {
        r++;
        re = hr.pre[r + 1];
        have = false;
      }
      if (!have) {
        const int32_t v = hr.hi[hr.huge[r]];
        x0 = g.xadj[v] - hr.pre[r];
        p = pi[v];
        have = true;
      }
      const int64_t e = x0 + f;
      acc += (int64_t)g.adjw[e] * dcode(sdist, p, pi[g.adj[e]]);
    }
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)Jacc, (unsigned long long)acc);
}

// ---------------------------------------------------------------------------
// Alg. 4 step 1: best target per vertex by Eq. 1, non-negative filter
// ---------------------------------------------------------------------------
// Best target of one vertex: argmin over the neighbouring PEs q != p of
// T(q) = sum_j w_j D(q, c_j) (ties: lowest code), i.e. argmax of Eq. 1's
// G_q(v) = T(p) - T(q).  Returns false if no neighbour lies outside p.
template <class Row>
__device__ __forceinline__ bool best_target(const Row& r, int deg, int32_t p, const int32_t* sdist, int32_t& best_c,
                                            int64_t& best_T) {
  best_c = INT32_MAX;
  best_T = INT64_MAX;
  bool any = false;
  for (int j = 0; j < deg; j++) {
    const int32_t q = r.code(j);
    if (q == p) continue;
    bool seen = false;
    for (int l = 0; l < j; l++)
      if (r.code(l) == q) {
        seen = true;
        break;
      }
    if (seen) continue;
    any = true;
    const int64_t T = row_cost(r, deg, sdist, q);
    if (T < best_T || (T == best_T && q < best_c)) {
      best_T = T;
      best_c = q;
    }
  }
  return any;
}

// Alg. 4 filter: G >= 0, or with the relaxed filter (relax_num > 0) also
// -G < floor(relax_num conn(v, P(v)) / relax_den).
struct LpFilter {
  int32_t num, den;
  __device__ __forceinline__ bool admit(int64_t G, int64_t own) const {
    return G >= 0 || (num > 0 && -G < ((int64_t)num * own) / den);
  }
};

// weight of a row's entries inside PE p
template <class Row>
__device__ __forceinline__ int64_t row_own(const Row& r, int deg, int32_t p) {
  int64_t s = 0;
  for (int j = 0; j < deg; j++) s += r.code(j) == p ? r.weight(j) : 0;
  return s;
}

// Sub-warp work queue of a staged tile: the lanes in `work` (vertices with a
// neighbour outside their own PE) are served four at a time by 8-lane
// sub-warps; each sub-warp evaluates T(q) for every distinct neighbouring PE
// q != p of its vertex from the staged entries and keeps the minimum (lowest
// code on ties).  out(lane, G = T(p) - T(q*), q*, p, conn(v, p)) runs on the
// sub-warp's first lane; conn(v, p) is summed only when `own` is set (else 0).
// In a tile whose range was not staged (it exceeds the buffer capacity
// `cap`), each sub-warp first copies its vertex's row into its quarter of
// the buffer with `load`.
struct RowLoader {
  const int32_t* __restrict__ adj;
  const int32_t* __restrict__ adjw;
  const int32_t* __restrict__ pi;
  __device__ __forceinline__ void operator()(int64_t vb, int dg, int sl, int32_t* c, int32_t* w) const {
    for (int j = sl; j < dg; j += kSubWarp) {
      c[j] = pi[adj[vb + j]];
      w[j] = adjw[vb + j];
    }
  }
};
struct NoRowLoader {  // callers that never queue a vertex of an unstaged tile
  __device__ __forceinline__ void operator()(int64_t, int, int, int32_t*, int32_t*) const {}
};

template <class Load, class Out>
__device__ __forceinline__ void tile_gain_queue(unsigned work, const TileLane& t, int32_t p, int64_t Tp,
                                                int32_t* sc, int32_t* sw, int cap, Load load,
                                                const int32_t* sdist, int lane, bool own, Out out) {
  const int sub = lane >> 3, sl = lane & 7;
  const int rounds = (__popc(work) + 3) / 4;
  for (int r = 0; r < rounds; r++) {
    const int src = tile_worker(work, r, sub);
    const int s2 = src < 0 ? 0 : src;
    const int64_t vb = __shfl_sync(0xffffffffu, t.b, s2);
    const int dg = (int)(__shfl_sync(0xffffffffu, t.e, s2) - vb);
    const int32_t pv = __shfl_sync(0xffffffffu, p, s2);
    const int64_t tp = __shfl_sync(0xffffffffu, Tp, s2);
    int64_t off = vb - t.E0;
    if (!t.staged) {  // warp-uniform
      off = sub * (cap / 4);
      __syncwarp();  // the previous round has read this quarter
      if (src >= 0) load(vb, dg, sl, sc + off, sw + off);
      __syncwarp();
    }
    const int32_t* c = sc + off;
    const int32_t* w = sw + off;
    int64_t bt = INT64_MAX, ow = 0;
    int32_t bc = INT32_MAX;
    if (src >= 0) {
      for (int j = sl; j < dg; j += kSubWarp) {
        const int32_t q = c[j];
        if (q == pv) {
          ow += w[j];
          continue;
        }
        int64_t T = 0;
        for (int l = 0; l < dg; l++) T += (int64_t)w[l] * dcode(sdist, q, c[l]);
        if (T < bt || (T == bt && q < bc)) {
          bt = T;
          bc = q;
        }
      }
    }
#pragma unroll
    for (int o = kSubWarp / 2; o > 0; o >>= 1) {
      const int64_t ot = __shfl_xor_sync(0xffffffffu, bt, o);
      const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (ot < bt || (ot == bt && oc < bc)) {
        bt = ot;
        bc = oc;
      }
      if (own) ow += __shfl_xor_sync(0xffffffffu, ow, o);
    }
    if (src >= 0 && sl == 0) out(src, tp - bt, bc, pv, ow);
  }
}

// Alg. 4 step 1 for the low-degree vertices.  Warp tiles stage the
// neighbour PEs; each lane checks its own vertex (T(P(v)), any neighbour
// outside P(v)); the vertices with candidates are then evaluated four at a
// time by 8-lane sub-warps from the staged entries (in a tile too long to
// stage, from the row each sub-warp copies into shared memory first).
__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks) k_lp_gain_tile(GraphView g, const int32_t* __restrict__ pi,
                                                               uint8_t* __restrict__ lock, int32_t* __restrict__ pp,
                                                               int64_t* __restrict__ gain, uint8_t* __restrict__ inx,
                                                               Topo topo, LpFilter flt, const RefineState* st) {
  __shared__ int32_t sdist[32];
  __shared__ int32_t sc[kTileWarps][kTileE];
  __shared__ int32_t sw[kTileWarps][kTileE];
  if (!kind_is(st, 1 << KIND_LP)) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileGraph tg{g.n, g.xadj, g.adj, g.adjw};
  const int64_t ntiles = ((int64_t)g.n + kTileV - 1) / kTileV;
  for (int64_t tile = (int64_t)blockIdx.x * kTileWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kTileWarps) {
    const TileLane t = stage_tile(tg, tile * kTileV, lane, sc[warp], sw[warp], GatherPi{pi});
    const int deg = (int)(t.e - t.b);
    const bool low = t.v < g.n && deg <= kLowDeg;
    int32_t p = -1;
    int64_t Tp = 0;
    bool cand = false;
    if (low) {
      p = pi[t.v];
      if (lock[t.v]) {
        lock[t.v] = 0;
      } else if (t.staged) {
        // T(P(v)) only for vertices with a neighbour outside P(v): interior
        // vertices (most of them on a refined level) skip the distance sum
        const int32_t* c = sc[warp] + (t.b - t.E0);
        const int32_t* w = sw[warp] + (t.b - t.E0);
        for (int j = 0; j < deg; j++) cand |= c[j] != p;
        if (cand)
          for (int j = 0; j < deg; j++) Tp += (int64_t)w[j] * dcode(sdist, p, c[j]);
      } else {  // oversized tile: the lane check from global memory; a sub-warp stages the row below
        for (int j = 0; j < deg; j++) {
          const int32_t q = pi[g.adj[t.b + j]];
          cand |= q != p;
          Tp += (int64_t)g.adjw[t.b + j] * dcode(sdist, p, q);
        }
      }
      if (!cand) {  // locked, or no neighbour outside P(v)
        inx[t.v] = 0;
        pp[t.v] = p;
        gain[t.v] = 0;
      }
    }
    const unsigned work = __ballot_sync(0xffffffffu, cand);
    tile_gain_queue(work, t, p, Tp, sc[warp], sw[warp], kTileE, RowLoader{g.adj, g.adjw, pi}, sdist, lane,
                    flt.num > 0,
                    [&](int src, int64_t G, int32_t bc, int32_t pv, int64_t own) {
                      const int64_t v = tile * kTileV + src;
                      const bool in = flt.admit(G, own);
                      inx[v] = in ? 1 : 0;
                      pp[v] = in ? bc : pv;
                      gain[v] = in ? G : 0;
                    });
    __syncwarp();
  }
}

// Shared-memory layout of the dense connectivity array and its group sums.
struct GroupLayout {
  int32_t off[kMaxLevels + 1];  // off[0] = 0 (conn itself), off[i] = start of level-i group sums
  int32_t total;
};
__host__ inline GroupLayout group_layout(const Topo& t) {
  GroupLayout gl{};
  int32_t o = t.kc;
  gl.off[0] = 0;
  for (int i = 1; i <= t.levels; i++) {
    gl.off[i] = o;
    o += t.kc >> t.s[i];
  }
  gl.total = o;
  return gl;
}

// Fills conn[0, kc) (already zeroed) with the edge weights of v per neighbour
// PE and the level group sums after it.  Returns T(P(v)) summed over the block.
// conn of the CSR entries [e0, e1) added into tab[code] (shared memory):
// four entries per thread at a time, whose adjacency loads and PE gathers
// are all issued before the first add.
__device__ __forceinline__ void conn_add(const GraphView& g, int64_t e0, int64_t e1, const int32_t* __restrict__ pi,
                                         int32_t* tab) {
  constexpr int kB = 4;
  const int64_t step = blockDim.x;
  int64_t e = e0 + threadIdx.x;
  for (; e + (kB - 1) * step < e1; e += kB * step) {
    int32_t u[kB], w[kB];
#pragma unroll
    for (int b = 0; b < kB; b++) {
      u[b] = g.adj[e + b * step];
      w[b] = g.adjw[e + b * step];
    }
#pragma unroll
    for (int b = 0; b < kB; b++) u[b] = pi[u[b]];
#pragma unroll
    for (int b = 0; b < kB; b++) atomicAdd(&tab[u[b]], w[b]);
  }
  for (; e < e1; e += step) atomicAdd(&tab[pi[g.adj[e]]], g.adjw[e]);
}

// The level group sums of a complete conn table (layout of GroupLayout).
__device__ void conn_groups(const Topo& topo, const GroupLayout& gl, int32_t* tab) {
  for (int i = 1; i <= topo.levels; i++) {
    const int32_t cnt = topo.kc >> topo.s[i];
    const int32_t sh = topo.s[i] - topo.s[i - 1];
    const int32_t* prev = tab + gl.off[i - 1];
    int32_t* cur = tab + gl.off[i];
    for (int32_t gidx = threadIdx.x; gidx < cnt; gidx += blockDim.x) {
      int32_t s = 0;
      for (int32_t j = 0; j < (1 << sh); j++) s += prev[(gidx << sh) + j];
      cur[gidx] = s;
    }
    __syncthreads();
  }
}

__device__ void conn_build(const GraphView& g, int32_t v, const int32_t* __restrict__ pi, const Topo& topo,
                           const GroupLayout& gl, int32_t* tab) {
  conn_add(g, g.xadj[v], g.xadj[v + 1], pi, tab);
  __syncthreads();
  conn_groups(topo, gl, tab);
}

// sum_b conn(b) D(q, b) from the group sums (Eq. 1 regrouped by level).
__device__ __forceinline__ int64_t conn_T(const int32_t* tab, const Topo& topo, const GroupLayout& gl, int32_t q) {
  int64_t T = 0;
  int32_t prev = tab[q];
  for (int i = 1; i <= topo.levels; i++) {
    const int32_t cur = tab[gl.off[i] + (q >> topo.s[i])];
    T += (int64_t)topo.dist[i - 1] * (cur - prev);
    prev = cur;
  }
  return T;
}

// Alg. 4 step 1 for vertex v (current PE code p) from its complete table
// (conn over the PE codes and the level group sums): the neighbouring PE
// q != p of smallest T(q) (lowest code on ties), the filter, the outputs.
// All threads of the CTA call it; ends with a barrier.
__device__ __forceinline__ void lp_hub_decide(const int32_t* tab, const Topo& topo, const GroupLayout& gl,
                                              const LpFilter& flt, int32_t v, int32_t p, int32_t* pp, int64_t* gain,
                                              uint8_t* inx, int64_t* sbt, int32_t* sbc) {
  int64_t bt = INT64_MAX;
  int32_t bc = INT32_MAX;
  for (int32_t q = threadIdx.x; q < topo.kc; q += blockDim.x) {
    if (q == p || tab[q] == 0) continue;
    const int64_t T = conn_T(tab, topo, gl, q);
    if (T < bt || (T == bt && q < bc)) {
      bt = T;
      bc = q;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t ot = __shfl_xor_sync(0xffffffffu, bt, o);
    const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
    if (ot < bt || (ot == bt && oc < bc)) {
      bt = ot;
      bc = oc;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sbt[threadIdx.x >> 5] = bt;
    sbc[threadIdx.x >> 5] = bc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++)
      if (sbt[w] < bt || (sbt[w] == bt && sbc[w] < bc)) {
        bt = sbt[w];
        bc = sbc[w];
      }
    const int64_t Tp = conn_T(tab, topo, gl, p);
    const int64_t G = Tp - bt;
    if (bc != INT32_MAX && flt.admit(G, tab[p])) {
      inx[v] = 1;
      pp[v] = bc;
      gain[v] = G;
    } else {
      inx[v] = 0;
      pp[v] = p;
      gain[v] = 0;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kHiThreads) k_lp_gain_high(GraphView g, const int32_t* __restrict__ hi,
                                                             const int32_t* __restrict__ sel, int32_t n_sel,
                                                             const int32_t* __restrict__ pi, uint8_t* lock,
                                                             int32_t* pp, int64_t* gain, uint8_t* inx, Topo topo,
                                                             GroupLayout gl, LpFilter flt, const RefineState* st) {
  extern __shared__ int32_t tab[];
  __shared__ int64_t sbt[32];
  __shared__ int32_t sbc[32];
  if (!kind_is(st, 1 << KIND_LP)) return;
  for (int32_t i = blockIdx.x; i < n_sel; i += gridDim.x) {
    const int32_t v = hi_vertex(hi, sel, i);
    const int32_t p = pi[v];
    if (lock[v]) {
      __syncthreads();
      if (threadIdx.x == 0) {
        inx[v] = 0;
        pp[v] = p;
        gain[v] = 0;
        lock[v] = 0;
      }
      continue;
    }
    for (int32_t b = threadIdx.x; b < gl.total; b += blockDim.x) tab[b] = 0;
    __syncthreads();
    conn_build(g, v, pi, topo, gl, tab);
    lp_hub_decide(tab, topo, gl, flt, v, p, pp, gain, inx, sbt, sbc);
  }
}

// Per-warp dense connectivity table of one mid-degree vertex: each lane's
// entries (PE codes q[r], weights w[r]; q < 0 for none) are added to conn at
// ct[q] and, with `groups`, to the level group sums ct[off_i + (q >> s_i)]
// (the layout of conn_build), by shared-memory atomics.  With `add` false it
// undoes that (stores zeros at the same slots) once the table has been read.
__device__ __forceinline__ void mid_table(int32_t* ct, const int32_t (&q)[kMidPer], const int32_t (&w)[kMidPer],
                                          const Topo& topo, const GroupLayout& gl, bool groups, bool add) {
#pragma unroll
  for (int r = 0; r < kMidPer; r++) {
    if (q[r] < 0) continue;
    if (add) atomicAdd(&ct[q[r]], w[r]);
    else ct[q[r]] = 0;
    if (groups)
      for (int i = 1; i <= topo.levels; i++) {
        int32_t* slot = &ct[gl.off[i] + (q[r] >> topo.s[i])];
        if (add) atomicAdd(slot, w[r]);
        else *slot = 0;
      }
  }
}

// Loads a mid-degree row into registers: PE codes of the neighbours (-1 past
// the row) and edge weights; all loads of a stage are issued before any use.
__device__ __forceinline__ void mid_row(const GraphView& g, const int32_t* __restrict__ pi, int64_t beg, int64_t deg,
                                        int lane, int32_t (&q)[kMidPer], int32_t (&w)[kMidPer]) {
#pragma unroll
  for (int r = 0; r < kMidPer; r++) {
    const int j = lane + 32 * r;
    q[r] = j < deg ? g.adj[beg + j] : -1;
    w[r] = j < deg ? g.adjw[beg + j] : 0;
  }
#pragma unroll
  for (int r = 0; r < kMidPer; r++) q[r] = q[r] >= 0 ? pi[q[r]] : -1;
}

// Alg. 4 step 1 for the vertices of degree in (kLowDeg, kMidDeg]: one warp
// per vertex with its own dense table (conn and level group sums) in shared
// memory; the candidates are the PEs of the row's entries (conn > 0), so the
// argmin of T over them equals k_lp_gain_high's scan of the code space.
__global__ void __launch_bounds__(kMidThreads) k_lp_gain_mid(GraphView g, const int32_t* __restrict__ hi, int32_t n_hi,
                                                             const int32_t* __restrict__ pi, uint8_t* lock,
                                                             int32_t* pp, int64_t* gain, uint8_t* inx, Topo topo,
                                                             GroupLayout gl, LpFilter flt, const RefineState* st) {
  extern __shared__ int32_t mtab[];
  if (!kind_is(st, 1 << KIND_LP)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* ct = mtab + (int64_t)warp * gl.total;
  for (int32_t b = lane; b < gl.total; b += 32) ct[b] = 0;
  __syncwarp();
  for (int64_t i = (int64_t)blockIdx.x * kMidWarps + warp; i < n_hi; i += (int64_t)gridDim.x * kMidWarps) {
    const int32_t v = hi[i];
    const int64_t beg = g.xadj[v];
    const int64_t deg = g.xadj[v + 1] - beg;
    if (deg > g.mid_deg) continue;
    const int32_t p = pi[v];
    const bool locked = lock[v] != 0;
    __syncwarp();  // every lane has read the lock before lane 0 clears it
    if (locked) {
      if (lane == 0) {
        inx[v] = 0;
        pp[v] = p;
        gain[v] = 0;
        lock[v] = 0;
      }
      continue;
    }
    int32_t q[kMidPer], w[kMidPer];
    mid_row(g, pi, beg, deg, lane, q, w);
    mid_table(ct, q, w, topo, gl, true, true);
    __syncwarp();
    int64_t bt = INT64_MAX;
    int32_t bc = INT32_MAX;
#pragma unroll
    for (int r = 0; r < kMidPer; r++) {
      if (q[r] < 0 || q[r] == p) continue;
      const int64_t T = conn_T(ct, topo, gl, q[r]);
      if (T < bt || (T == bt && q[r] < bc)) {
        bt = T;
        bc = q[r];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t ot = __shfl_xor_sync(0xffffffffu, bt, o);
      const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (ot < bt || (ot == bt && oc < bc)) {
        bt = ot;
        bc = oc;
      }
    }
    const int64_t Tp = conn_T(ct, topo, gl, p);
    const int64_t own = ct[p];
    __syncwarp();
    mid_table(ct, q, w, topo, gl, true, false);
    __syncwarp();
    if (lane == 0) {
      const int64_t G = bc != INT32_MAX ? Tp - bt : 0;
      if (bc != INT32_MAX && flt.admit(G, own)) {
        inx[v] = 1;
        pp[v] = bc;
        gain[v] = G;
      } else {
        inx[v] = 0;
        pp[v] = p;
        gain[v] = 0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Alg. 4 step 2: gain under the approximate future state given by ord
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t future_block(int32_t u, int32_t v, int64_t gv, const int32_t* __restrict__ pi,
                                                const int32_t* __restrict__ pp, const int64_t* __restrict__ gain,
                                                const uint8_t* __restrict__ inx) {
  if (inx[u]) {
    const int64_t gu = gain[u];
    if (gu > gv || (gu == gv && u < v)) return pp[u];
  }
  return pi[u];
}

__global__ void __launch_bounds__(kThreads) k_lp_after_low(GraphView g, const int32_t* __restrict__ pi,
                                                           const int32_t* __restrict__ pp,
                                                           const int64_t* __restrict__ gain,
                                                           const uint8_t* __restrict__ inx, uint8_t* lock, Topo topo,
                                                           const RefineState* st) {
  __shared__ int32_t sdist[32];
  if (!kind_is(st, 1 << KIND_LP)) return;
  load_sdist(sdist, topo);
  __syncthreads();
  auto tile = cg::tiled_partition<kSubWarp>(cg::this_thread_block());
  const int lane = tile.thread_rank();
  const int64_t nsw = ((int64_t)gridDim.x * blockDim.x) / kSubWarp;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kSubWarp; v < g.n; v += nsw) {
    if (!inx[v]) continue;
    const int64_t beg = g.xadj[v], end = g.xadj[v + 1];
    if (end - beg > kLowDeg) continue;
    const int32_t p = pi[v], q = pp[v];
    const int64_t gv = gain[v];
    int64_t s = 0;
    for (int64_t e = beg + lane; e < end; e += kSubWarp) {
      const int32_t b = future_block(g.adj[e], (int32_t)v, gv, pi, pp, gain, inx);
      s += (int64_t)g.adjw[e] * (dcode(sdist, p, b) - dcode(sdist, q, b));
    }
    s = tile_sum64(tile, s);
    if (lane == 0 && s >= 0) lock[v] = 1;
  }
}

// Alg. 4 step 2 for the vertices of degree in (kLowDeg, kMidDeg], one warp per vertex.
__global__ void __launch_bounds__(kMidThreads) k_lp_after_mid(GraphView g, const int32_t* __restrict__ hi, int32_t n_hi,
                                                              const int32_t* __restrict__ pi,
                                                              const int32_t* __restrict__ pp,
                                                              const int64_t* __restrict__ gain,
                                                              const uint8_t* __restrict__ inx, uint8_t* lock,
                                                              Topo topo, const RefineState* st) {
  __shared__ int32_t sdist[32];
  if (!kind_is(st, 1 << KIND_LP)) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)blockIdx.x * kMidWarps + warp; i < n_hi; i += (int64_t)gridDim.x * kMidWarps) {
    const int32_t v = hi[i];
    if (!inx[v]) continue;
    const int64_t beg = g.xadj[v], end = g.xadj[v + 1];
    if (end - beg > g.mid_deg) continue;
    const int32_t p = pi[v], q = pp[v];
    const int64_t gv = gain[v];
    int64_t s = 0;
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int32_t b = future_block(g.adj[e], v, gv, pi, pp, gain, inx);
      s += (int64_t)g.adjw[e] * (dcode(sdist, p, b) - dcode(sdist, q, b));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && s >= 0) lock[v] = 1;
  }
}

// Alg. 4 step 2 for the vertices of degree > kMidDeg in X: their entries,
// flattened in huge[] order, in chunks drawn by the CTAs of one wave; each
// chunk adds its part of a row's recomputed gain into the row's accumulator,
// and k_lp_after_hub_finish sets the locks (the moves that stay
// non-negative) and clears the accumulators.
__global__ void __launch_bounds__(kHiThreads) k_lp_after_hub(GraphView g, HubRows hr, const int32_t* __restrict__ pi,
                                                             const int32_t* __restrict__ pp,
                                                             const int64_t* __restrict__ gain,
                                                             const uint8_t* __restrict__ inx, int64_t* acc, Topo topo,
                                                             const RefineState* st, unsigned long long* ctr) {
  static_assert(kHiThreads == kSpanRows, "one thread per row of a span");
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  __shared__ int64_t s_ch;
  // the candidates among the rows of the current span, found at once
  __shared__ int32_t s_v[kSpanRows];  // -1: not a candidate
  __shared__ int64_t s_rb[kSpanRows], s_re[kSpanRows];
  if (!kind_is(st, 1 << KIND_LP)) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int64_t m_hub = hr.pre[hr.n_huge];
  const int64_t nspans = (hr.nchunks + kSpanChunks - 1) / kSpanChunks;
  for (int64_t sp = next_chunk(ctr, &s_ch); sp < nspans; sp = next_chunk(ctr, &s_ch)) {
    const int64_t cb = sp * kSpanChunks * kHubChunk, ce = min(cb + kSpanChunks * kHubChunk, m_hub);
    const int32_t r0 = hr.chunk[sp * kSpanChunks];
    const int32_t r = r0 + (int32_t)threadIdx.x;
    bool row = false;
    int32_t v = -1;
    int64_t rb = 0, re = 0;
    if (r < hr.n_huge) {
      rb = hr.pre[r];
      re = hr.pre[r + 1];
      row = rb < ce;
    }
    if (row) {
      const int32_t u = hr.hi[hr.huge[r]];
      if (inx[u]) v = u;
    }
    s_v[threadIdx.x] = v;
    s_rb[threadIdx.x] = rb;
    s_re[threadIdx.x] = re;
    const int nrows = __syncthreads_count(row);  // the span's rows are a prefix
    for (int i = 0; i < nrows; i++) {
      const int32_t w = s_v[i];
      if (w < 0) continue;
      const int32_t p = pi[w], q = pp[w];
      const int64_t gv = gain[w];
      const int64_t x0 = g.xadj[w] - s_rb[i];
      const int64_t f1 = min(s_re[i], ce);
      int64_t s = 0;
      for (int64_t f = max(s_rb[i], cb) + threadIdx.x; f < f1; f += blockDim.x) {
        const int64_t e = x0 + f;
        const int32_t b = future_block(g.adj[e], w, gv, pi, pp, gain, inx);
        s += (int64_t)g.adjw[e] * (dcode(sdist, p, b) - dcode(sdist, q, b));
      }
      s = block_sum(s, sm);
      if (threadIdx.x == 0 && s) atomicAdd((unsigned long long*)&acc[r0 + i], (unsigned long long)s);
    }
  }
  leave_chunks(ctr);
}

__global__ void k_lp_after_hub_finish(HubRows hr, const uint8_t* __restrict__ inx, int64_t* acc, uint8_t* lock,
                                      const RefineState* st) {
  if (!kind_is(st, 1 << KIND_LP)) return;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < hr.n_huge; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = hr.hi[hr.huge[r]];
    if (!inx[v]) continue;
    if (acc[r] >= 0) lock[v] = 1;
    acc[r] = 0;
  }
}

// ---------------------------------------------------------------------------
// Exact change of J by a simultaneous move (LP step 3, weak rebalancing)
// ---------------------------------------------------------------------------
// With M the movers, J changes by the sum over the CSR entries (v, u) of the
// movers' rows of w (D(new v, new u) - D(old v, old u)), doubled when u stays
// (the entry (u, v) of u's row changes by the same amount but u's row is not
// visited) and taken once when u moves too (its own row adds the twin entry).
// Launched before the move is applied (P still holds the old mapping).
struct LpMoves {  // LP: M = lock, target P'
  const uint8_t* lock;
  const int32_t* pp;
  __device__ __forceinline__ bool moved(int64_t v) const { return lock[v] != 0; }
  __device__ __forceinline__ int32_t target(int64_t v) const { return pp[v]; }
};
struct WeakMoves {  // weak rebalancing: M = eligible and selected, target the destination
  const uint8_t* elig;
  const uint8_t* sel;
  const int32_t* dest;
  __device__ __forceinline__ bool moved(int64_t v) const { return elig[v] && sel[v]; }
  __device__ __forceinline__ int32_t target(int64_t v) const { return dest[v]; }
};

template <class Mv>
__device__ __forceinline__ int64_t delta_entry(const Mv& mv, const int32_t* pi, const int32_t* sdist,
                                               int32_t ov, int32_t nv, int32_t u, int32_t w) {
  const int32_t ou = pi[u];
  const bool um = mv.moved(u);
  const int32_t nu = um ? mv.target(u) : ou;
  const int64_t d = (int64_t)w * (dcode(sdist, nv, nu) - dcode(sdist, ov, ou));
  return um ? d : 2 * d;
}

// movers of degree <= kLowDeg: one 8-lane sub-warp per vertex
template <class Mv>
__global__ void __launch_bounds__(kThreads) k_delta_low(GraphView g, const int32_t* __restrict__ pi, Mv mv, Topo topo,
                                                        int64_t* Jacc, const RefineState* st, int kind) {
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  if (st->kind != kind) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int lane = threadIdx.x & (kSubWarp - 1);
  const int64_t nsw = ((int64_t)gridDim.x * blockDim.x) / kSubWarp;
  int64_t acc = 0;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kSubWarp; v < g.n; v += nsw) {
    if (!mv.moved(v)) continue;
    const int64_t b = g.xadj[v], e = g.xadj[v + 1];
    if (e - b > kLowDeg) continue;
    const int32_t ov = pi[v], nv = mv.target(v);
    for (int64_t x = b + lane; x < e; x += kSubWarp) acc += delta_entry(mv, pi, sdist, ov, nv, g.adj[x], g.adjw[x]);
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)Jacc, (unsigned long long)acc);
}

// movers of degree in (kLowDeg, kMidDeg]: one warp per vertex
template <class Mv>
__global__ void __launch_bounds__(kMidThreads) k_delta_mid(GraphView g, const int32_t* __restrict__ hi, int32_t n_hi,
                                                           const int32_t* __restrict__ pi, Mv mv, Topo topo,
                                                           int64_t* Jacc, const RefineState* st, int kind) {
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  if (st->kind != kind) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * kMidWarps + warp; i < n_hi; i += (int64_t)gridDim.x * kMidWarps) {
    const int32_t v = hi[i];
    if (!mv.moved(v)) continue;
    const int64_t b = g.xadj[v], e = g.xadj[v + 1];
    if (e - b > g.mid_deg) continue;
    const int32_t ov = pi[v], nv = mv.target(v);
    for (int64_t x = b + lane; x < e; x += 32) acc += delta_entry(mv, pi, sdist, ov, nv, g.adj[x], g.adjw[x]);
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)Jacc, (unsigned long long)acc);
}

// movers of degree > kMidDeg: the flattened hub entries in chunks of
// kHubChunk over the CTAs of one wave (as k_eval_high); the entries of rows
// that do not move are skipped
template <class Mv>
__global__ void __launch_bounds__(kHiThreads) k_delta_high(GraphView g, HubRows hr, const int32_t* __restrict__ pi,
                                                           Mv mv, Topo topo, int64_t* Jacc, const RefineState* st,
                                                           int kind) {
  static_assert(kHiThreads == kSpanRows, "one thread per row of a span");
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  // the movers among the rows of the current span, found at once
  __shared__ int32_t s_v[kSpanRows];  // -1: the row stays
  __shared__ int64_t s_rb[kSpanRows], s_re[kSpanRows];
  if (st->kind != kind) return;
  load_sdist(sdist, topo);
  __syncthreads();
  const int64_t m_hub = hr.pre[hr.n_huge];
  const int64_t nspans = (hr.nchunks + kSpanChunks - 1) / kSpanChunks;
  int64_t acc = 0;
  for (int64_t sp = blockIdx.x; sp < nspans; sp += gridDim.x) {
    const int64_t cb = sp * kSpanChunks * kHubChunk, ce = min(cb + kSpanChunks * kHubChunk, m_hub);
    const int32_t r = hr.chunk[sp * kSpanChunks] + (int32_t)threadIdx.x;
    bool row = false;
    int32_t v = -1;
    int64_t rb = 0, re = 0;
    if (r < hr.n_huge) {
      rb = hr.pre[r];
      re = hr.pre[r + 1];
      row = rb < ce;
    }
    if (row) {
      const int32_t u = hr.hi[hr.huge[r]];
      if (mv.moved(u)) v = u;
    }
    s_v[threadIdx.x] = v;
    s_rb[threadIdx.x] = rb;
    s_re[threadIdx.x] = re;
    const int nrows = __syncthreads_count(row);  // the span's rows are a prefix
    for (int i = 0; i < nrows; i++) {
      const int32_t w = s_v[i];
      if (w < 0) continue;
      const int64_t x0 = g.xadj[w] - s_rb[i];  // CSR position of flat entry f: x0 + f
      const int32_t ov = pi[w], nv = mv.target(w);
      const int64_t f1 = min(s_re[i], ce);
      for (int64_t f = max(s_rb[i], cb) + threadIdx.x; f < f1; f += blockDim.x) {
        const int64_t e = x0 + f;
        acc += delta_entry(mv, pi, sdist, ov, nv, g.adj[e], g.adjw[e]);
      }
    }
    __syncthreads();  // the row table is rewritten for the next span
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)Jacc, (unsigned long long)acc);
}

// Alg. 4 step 3: simultaneous move of M (lock = moved), block weights.
// Block-weight changes of a simultaneous move.  With a PE code space of at
// most kApplyCodes codes each CTA sums its changes in shared memory and adds
// the non-zero ones to W at the end: movers crowd into a few blocks (a hub's
// neighbourhood moves together on power-law graphs), and one global atomic per
// mover on the same few words serialises.
constexpr int32_t kApplyCodes = 4096;
struct BlockDelta {
  long long* dW;  // shared, kApplyCodes
  int64_t* W;
  bool local;
  __device__ __forceinline__ void init(int32_t kc) {
    if (local)
      for (int32_t b = threadIdx.x; b < kc; b += blockDim.x) dW[b] = 0;
  }
  __device__ __forceinline__ void move(int32_t p, int32_t q, int64_t c) {
    if (local) {
      atomicAdd((unsigned long long*)&dW[p], (unsigned long long)(-c));
      atomicAdd((unsigned long long*)&dW[q], (unsigned long long)c);
    } else {
      atomicAdd((unsigned long long*)&W[p], (unsigned long long)(-c));
      atomicAdd((unsigned long long*)&W[q], (unsigned long long)c);
    }
  }
  // after a barrier
  __device__ __forceinline__ void flush(int32_t kc) {
    if (local)
      for (int32_t b = threadIdx.x; b < kc; b += blockDim.x)
        if (dW[b]) atomicAdd((unsigned long long*)&W[b], (unsigned long long)dW[b]);
  }
};

__global__ void __launch_bounds__(kThreads) k_lp_apply(int32_t n, int32_t* __restrict__ pi,
                                                       const int32_t* __restrict__ pp,
                                                       const uint8_t* __restrict__ lock,
                                                       const int32_t* __restrict__ vw, int64_t* W, int32_t kc,
                                                       RefineState* st) {
  __shared__ int32_t cnt;
  __shared__ long long dW[kApplyCodes];
  if (!kind_is(st, 1 << KIND_LP)) return;
  BlockDelta bd{dW, W, kc <= kApplyCodes};
  bd.init(kc);
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int32_t mine = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!lock[v]) continue;
    const int32_t p = pi[v], q = pp[v];
    pi[v] = q;
    bd.move(p, q, vw[v]);
    mine++;
  }
  if (mine) atomicAdd(&cnt, mine);
  __syncthreads();
  bd.flush(kc);
  if (threadIdx.x == 0 && cnt) atomicAdd(&st->moved, cnt);
}

// ---------------------------------------------------------------------------
// rebalancing (Alg. 5, edge-cut loss; strong variant)
// ---------------------------------------------------------------------------
enum { CNT_NU = 0, CNT_SIGMA = 1, CNT_ELIG = 2, CNT_SEL = 3, CNT_TMP = 4, CNT_N = 8 };

struct RebPrepArgs {
  const int64_t* W;
  const int32_t* pe_of_code;
  Topo topo;
  int64_t lmax;
  int64_t cV;
  int32_t sigma_gap;
  int32_t* U;
  int64_t* cnt;
  int64_t* accepted;
};

// sigma, the fallback destination list U (ascending codes of valid PEs with
// weight <= sigma), and resets of the per-step counters (all threads).
__device__ void reb_prep_body(const RebPrepArgs& p, bool strong) {
  __shared__ int64_t sm[33];
  int64_t sigma;
  if (strong) {
    sigma = p.lmax;
  } else {
    const int64_t avg = (p.cV + p.topo.k - 1) / p.topo.k;
    sigma = p.lmax - p.sigma_gap;
    if (sigma < avg) sigma = avg;
  }
  int64_t carry = 0;
  for (int32_t base = 0; base < p.topo.kc; base += blockDim.x) {
    const int32_t b = base + threadIdx.x;
    const int64_t ok = (b < p.topo.kc && p.pe_of_code[b] >= 0 && p.W[b] <= sigma) ? 1 : 0;
    int64_t tot;
    const int64_t e = block_exclusive_scan(ok, sm, &tot);
    if (ok) p.U[carry + e] = b;
    carry += tot;
  }
  for (int32_t b = threadIdx.x; b < p.topo.kc; b += blockDim.x) p.accepted[b] = 0;
  if (threadIdx.x == 0) {
    p.cnt[CNT_NU] = carry;
    p.cnt[CNT_SIGMA] = sigma;
  }
}

__global__ void __launch_bounds__(1024) k_reb_prep(RebPrepArgs p, const RefineState* st) {
  if (!kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG))) return;
  reb_prep_body(p, st->kind == KIND_STRONG);
}

// Graph mode: the start of one Alg. 6 iteration selects the step bodies and,
// for a rebalancing step, prepares it.
__global__ void __launch_bounds__(1024) k_decide_prep(const RefineState* s, cudaGraphConditionalHandle h_lp,
                                                      cudaGraphConditionalHandle h_reb,
                                                      cudaGraphConditionalHandle h_strong, RebPrepArgs p) {
  const int32_t kind = s->kind;
  if (threadIdx.x == 0) {
    cudaGraphSetConditional(h_lp, kind == KIND_LP ? 1u : 0u);
    cudaGraphSetConditional(h_reb, (kind == KIND_WEAK || kind == KIND_STRONG) ? 1u : 0u);
    cudaGraphSetConditional(h_strong, kind == KIND_STRONG ? 1u : 0u);
  }
  if (kind == KIND_WEAK || kind == KIND_STRONG) reb_prep_body(p, kind == KIND_STRONG);
}

struct RebArgs {
  const int64_t* W;
  const int32_t* U;
  const int64_t* cnt;
  int64_t* tab;  // eligible weight per (source block, loss bucket)
  int64_t lmax;
  int64_t cV;
  int32_t k;
  uint64_t seed;
  int32_t obj;   // 0: cut gains conn(v, q) - conn(v, A); 1: Eq. 1 gains T(A) - T(q)
  Topo topo;     // distances for the J gains
};

__device__ __forceinline__ bool reb_eligible(const RebArgs& a, int32_t A, int32_t cv) {
  const int64_t WA = a.W[A];
  if (WA <= a.lmax) return false;
  // heavy: c(v) > 1.5 (c(A) - c(V)/k), in integers: 2k c(v) > 3 (k c(A) - c(V))
  return !(2 * (int64_t)a.k * cv > 3 * ((int64_t)a.k * WA - a.cV));
}

__global__ void __launch_bounds__(kThreads) k_reb_select_low(GraphView g, const int32_t* __restrict__ pi, RebArgs a,
                                                             int32_t* __restrict__ dest, uint8_t* __restrict__ bkt,
                                                             uint8_t* __restrict__ elig, const RefineState* st) {
  __shared__ int32_t sdist[32];
  if (!kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG))) return;
  if (a.obj) {
    load_sdist(sdist, a.topo);
    __syncthreads();
  }
  auto tile = cg::tiled_partition<kSubWarp>(cg::this_thread_block());
  const int lane = tile.thread_rank();
  const int wl = threadIdx.x & 31, sub = wl / kSubWarp;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t sigma = a.cnt[CNT_SIGMA];
  const int64_t nU = a.cnt[CNT_NU];
  const int32_t level = st->level, t = st->t;
  // 32 vertices per warp: each lane checks its vertex's eligibility (most
  // are not: their blocks are not overloaded), then the eligible ones are
  // served four at a time by the 8-lane sub-warps
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < g.n; base += nwarps * 32) {
    const int64_t vl = base + wl;
    bool want = false;
    int64_t beg_l = 0;
    int deg_l = 0;
    int32_t A_l = 0;
    if (vl < g.n) {
      beg_l = g.xadj[vl];
      deg_l = (int)(g.xadj[vl + 1] - beg_l);
      if (deg_l <= kLowDeg) {
        A_l = pi[vl];
        want = reb_eligible(a, A_l, g.vw[vl]);
        if (!want) elig[vl] = 0;
      }
    }
    const unsigned work = __ballot_sync(0xffffffffu, want);
    const int rounds = (__popc(work) + 3) / 4;
    for (int rnd = 0; rnd < rounds; rnd++) {
      const int src = tile_worker(work, rnd, sub);
      const int s2 = src < 0 ? 0 : src;
      const int64_t v = base + s2;
      const int64_t beg = __shfl_sync(0xffffffffu, beg_l, s2);
      const int deg = __shfl_sync(0xffffffffu, deg_l, s2);
      const int32_t A = __shfl_sync(0xffffffffu, A_l, s2);
      if (src < 0) continue;
      int32_t c[kSlots], w[kSlots];
      int32_t connA = 0;
#pragma unroll
      for (int r = 0; r < kSlots; r++) {
        const int idx = lane + kSubWarp * r;
        if (idx < deg) {
          c[r] = pi[g.adj[beg + idx]];
          w[r] = g.adjw[beg + idx];
        } else {
          c[r] = A;
          w[r] = 0;
        }
        if (c[r] == A) connA += w[r];
      }
      connA = tile_sum32(tile, connA);
      // score of each slot's block: conn(v, q), or -T(q) for the J gains (only
      // destinations below sigma are candidates)
      int64_t cc[kSlots];
#pragma unroll
      for (int r = 0; r < kSlots; r++) cc[r] = 0;
      const int rows = (deg + kSubWarp - 1) / kSubWarp;
      for (int rr = 0; rr < rows; rr++) {
        const int32_t crr = pick(c, rr);
        const int32_t wrr = pick(w, rr);
        for (int j = 0; j < kSubWarp; j++) {
          const int32_t cs = tile.shfl(crr, j);
          const int32_t ws = tile.shfl(wrr, j);
          if (a.obj) {
#pragma unroll
            for (int r = 0; r < kSlots; r++) cc[r] -= (int64_t)ws * dcode(sdist, c[r], cs);
          } else {
#pragma unroll
            for (int r = 0; r < kSlots; r++) cc[r] += (c[r] == cs) ? ws : 0;
          }
        }
      }
      bool found = false;
      int64_t bconn = 0;
      int32_t bc = INT32_MAX;
#pragma unroll
      for (int r = 0; r < kSlots; r++) {
        if (c[r] == A || a.W[c[r]] > sigma) continue;
        if (!found || cc[r] > bconn || (cc[r] == bconn && c[r] < bc)) {
          bconn = cc[r];
          bc = c[r];
          found = true;
        }
      }
#pragma unroll
      for (int o = kSubWarp / 2; o > 0; o >>= 1) {
        const int64_t ob = tile.shfl_xor(bconn, o);
        const int32_t oc = tile.shfl_xor(bc, o);
        const bool of = tile.shfl_xor(found, o);
        if (of && (!found || ob > bconn || (ob == bconn && oc < bc))) {
          bconn = ob;
          bc = oc;
          found = true;
        }
      }
      // the source block's score, and the drawn block's when no neighbour qualifies
      int64_t sA = connA, sR = 0;
      int32_t qr = -1;
      if (!found && nU > 0) qr = a.U[h_rebalance(a.seed, level, t, (int32_t)v) % (uint64_t)nU];
      if (a.obj) {
        int64_t pa = 0, pr = 0;
#pragma unroll
        for (int r = 0; r < kSlots; r++) {
          pa -= (int64_t)w[r] * dcode(sdist, A, c[r]);
          if (qr >= 0) pr -= (int64_t)w[r] * dcode(sdist, qr, c[r]);
        }
        sA = tile_sum64(tile, pa);
        sR = tile_sum64(tile, pr);
      }
      if (lane == 0) {
        int64_t gcut;
        if (found) {
          gcut = bconn - sA;
        } else if (qr >= 0) {
          bc = qr;
          gcut = sR - sA;
        } else {
          elig[v] = 0;
          continue;
        }
        const int32_t bk = loss_bucket(gcut);
        dest[v] = bc;
        bkt[v] = (uint8_t)bk;
        elig[v] = 1;
        atomicAdd((unsigned long long*)&a.tab[(int64_t)A * kBuckets + bk], (unsigned long long)(int64_t)g.vw[v]);
      }
    }
  }
}

// Alg. 5 destination for the vertices of degree in (kLowDeg, kMidDeg]: one
// warp per vertex with its own dense table in shared memory (conn per PE code,
// plus the level group sums for the J gains); candidates are the PEs of the
// row's entries, as in k_reb_select_high.
__global__ void __launch_bounds__(kMidThreads) k_reb_select_mid(GraphView g, const int32_t* __restrict__ hi, int32_t n_hi,
                                                                const int32_t* __restrict__ pi, RebArgs a, int32_t kc,
                                                                GroupLayout gl, int32_t* dest, uint8_t* bkt,
                                                                uint8_t* elig, const RefineState* st) {
  extern __shared__ int32_t mtab[];
  if (!kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG))) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t total = a.obj ? gl.total : kc;
  const bool groups = a.obj != 0;
  int32_t* ct = mtab + (int64_t)warp * total;
  for (int32_t b = lane; b < total; b += 32) ct[b] = 0;
  __syncwarp();
  const int64_t sigma = a.cnt[CNT_SIGMA];
  const int64_t nU = a.cnt[CNT_NU];
  for (int64_t i = (int64_t)blockIdx.x * kMidWarps + warp; i < n_hi; i += (int64_t)gridDim.x * kMidWarps) {
    const int32_t v = hi[i];
    const int64_t beg = g.xadj[v];
    const int64_t deg = g.xadj[v + 1] - beg;
    if (deg > g.mid_deg) continue;
    const int32_t A = pi[v];
    if (!reb_eligible(a, A, g.vw[v])) {
      if (lane == 0) elig[v] = 0;
      continue;
    }
    int32_t q[kMidPer], w[kMidPer];
    mid_row(g, pi, beg, deg, lane, q, w);
    mid_table(ct, q, w, a.topo, gl, groups, true);
    __syncwarp();
    // score: conn(v, q), or -T(q) for the J gains; -1 / INT64_MIN: none
    int64_t bconn = a.obj ? INT64_MIN : -1;
    int32_t bc = INT32_MAX;
#pragma unroll
    for (int r = 0; r < kMidPer; r++) {
      const int32_t b = q[r];
      if (b < 0 || b == A || a.W[b] > sigma) continue;
      const int64_t sc = a.obj ? -conn_T(ct, a.topo, gl, b) : (int64_t)ct[b];
      if (sc > bconn || (sc == bconn && b < bc)) {
        bconn = sc;
        bc = b;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t ob = __shfl_xor_sync(0xffffffffu, bconn, o);
      const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (ob > bconn || (ob == bconn && oc < bc)) {
        bconn = ob;
        bc = oc;
      }
    }
    int64_t gcut = 0;
    bool ok = true;
    if (lane == 0) {
      const int64_t sA = a.obj ? -conn_T(ct, a.topo, gl, A) : (int64_t)ct[A];
      if (bc != INT32_MAX) {
        gcut = bconn - sA;
      } else if (nU > 0) {
        bc = a.U[h_rebalance(a.seed, st->level, st->t, v) % (uint64_t)nU];
        gcut = (a.obj ? -conn_T(ct, a.topo, gl, bc) : 0) - sA;
      } else {
        ok = false;
      }
    }
    __syncwarp();
    mid_table(ct, q, w, a.topo, gl, groups, false);
    __syncwarp();
    if (lane == 0) {
      if (ok) {
        const int32_t bk = loss_bucket(gcut);
        dest[v] = bc;
        bkt[v] = (uint8_t)bk;
        atomicAdd((unsigned long long*)&a.tab[(int64_t)A * kBuckets + bk], (unsigned long long)(int64_t)g.vw[v]);
      }
      elig[v] = ok ? 1 : 0;
    }
  }
}

// Rebalancing selection for eligible vertex v of block A from its complete
// table (conn over the PE codes, plus the level group sums for the J gains):
// the best destination below sigma among the neighbouring blocks (the drawn
// block of U if none), its loss bucket, and the per-(block, bucket) weight
// totals.  All threads of the CTA call it; ends with a barrier.
__device__ __forceinline__ void reb_hub_decide(const int32_t* tab, const RebArgs& a, int32_t kc, const GroupLayout& gl,
                                               int32_t v, int32_t A, int32_t cv, int32_t* dest, uint8_t* bkt,
                                               uint8_t* elig, const RefineState* st, int64_t* sbb, int32_t* sbc) {
  const int64_t sigma = a.cnt[CNT_SIGMA];
  const int64_t nU = a.cnt[CNT_NU];
  // score: conn(v, q), or -T(q) for the J gains; -1 / INT64_MIN: none
  int64_t bconn = a.obj ? INT64_MIN : -1;
  int32_t bc = INT32_MAX;
  for (int32_t b = threadIdx.x; b < kc; b += blockDim.x) {
    const int32_t x = tab[b];
    if (x == 0 || b == A || a.W[b] > sigma) continue;
    const int64_t sc = a.obj ? -conn_T(tab, a.topo, gl, b) : (int64_t)x;
    if (sc > bconn || (sc == bconn && b < bc)) {
      bconn = sc;
      bc = b;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t ob = __shfl_xor_sync(0xffffffffu, bconn, o);
    const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
    if (ob > bconn || (ob == bconn && oc < bc)) {
      bconn = ob;
      bc = oc;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sbb[threadIdx.x >> 5] = bconn;
    sbc[threadIdx.x >> 5] = bc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++)
      if (sbb[w] > bconn || (sbb[w] == bconn && sbc[w] < bc)) {
        bconn = sbb[w];
        bc = sbc[w];
      }
    const int64_t sA = a.obj ? -conn_T(tab, a.topo, gl, A) : (int64_t)tab[A];
    int64_t gcut = 0;
    bool ok = true;
    if (bc != INT32_MAX) {
      gcut = bconn - sA;
    } else if (nU > 0) {
      bc = a.U[h_rebalance(a.seed, st->level, st->t, v) % (uint64_t)nU];
      gcut = (a.obj ? -conn_T(tab, a.topo, gl, bc) : 0) - sA;
    } else {
      ok = false;
    }
    if (ok) {
      const int32_t bk = loss_bucket(gcut);
      dest[v] = bc;
      bkt[v] = (uint8_t)bk;
      atomicAdd((unsigned long long*)&a.tab[(int64_t)A * kBuckets + bk], (unsigned long long)(int64_t)cv);
    }
    elig[v] = ok ? 1 : 0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kHiThreads) k_reb_select_high(GraphView g, const int32_t* __restrict__ hi,
                                                                const int32_t* __restrict__ sel, int32_t n_sel,
                                                                const int32_t* __restrict__ pi, RebArgs a, int32_t kc,
                                                                GroupLayout gl, int32_t* dest, uint8_t* bkt,
                                                                uint8_t* elig, const RefineState* st) {
  extern __shared__ int32_t tab[];  // conn per PE code (and the level group sums for the J gains)
  __shared__ int64_t sbb[32];
  __shared__ int32_t sbc[32];
  if (!kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG))) return;
  for (int32_t i = blockIdx.x; i < n_sel; i += gridDim.x) {
    const int32_t v = hi_vertex(hi, sel, i);
    const int32_t A = pi[v];
    if (!reb_eligible(a, A, g.vw[v])) {
      if (threadIdx.x == 0) elig[v] = 0;
      continue;
    }
    const int32_t total = a.obj ? gl.total : kc;
    for (int32_t b = threadIdx.x; b < total; b += blockDim.x) tab[b] = 0;
    __syncthreads();
    if (a.obj) {
      conn_build(g, v, pi, a.topo, gl, tab);
    } else {
      for (int64_t e = g.xadj[v] + threadIdx.x; e < g.xadj[v + 1]; e += blockDim.x)
        atomicAdd(&tab[pi[g.adj[e]]], g.adjw[e]);
      __syncthreads();
    }
    reb_hub_decide(tab, a, kc, gl, v, A, g.vw[v], dest, bkt, elig, st, sbb, sbc);
  }
}

// Connectivity-table kernels over the rows of degree > kMidDeg, spread over
// CTAs by chunk tickets (the table over the PE codes does not grow with the
// degree; the work does).  A row of at most split_deg entries is rated whole
// by the CTA that draws the chunk holding its first entry.  A larger row is
// rated in two launches: every chunk adds the conn of its entries into the
// row's global partial table, then one CTA per row reads the table back
// (emptying it), adds the level group sums and decides.  The policy P gives
// the table width, whether group sums are needed, which vertices take part
// and the decision.
struct LpHubPolicy {  // Alg. 4 step 1
  // skip() clears the lock that want() reads: a barrier between them
  static constexpr bool kWantBarrier = true;
  const int32_t* pi;
  uint8_t* lock;
  int32_t* pp;
  int64_t* gain;
  uint8_t* inx;
  Topo topo;
  GroupLayout gl;
  LpFilter flt;
  const RefineState* st;
  __device__ bool run() const { return kind_is(st, 1 << KIND_LP); }
  __device__ const Topo& topo_of() const { return topo; }
  __device__ int32_t topo_kc() const { return topo.kc; }
  __device__ int32_t words() const { return gl.total; }
  __device__ bool groups() const { return true; }
  __device__ bool want(int32_t v) const { return lock[v] == 0; }
  // a locked vertex keeps its PE, and its lock ends with this step
  __device__ void skip(int32_t v) const {
    inx[v] = 0;
    pp[v] = pi[v];
    gain[v] = 0;
    lock[v] = 0;
  }
  __device__ void decide(const int32_t* tab, int32_t v, int32_t cv, int64_t* sb, int32_t* sc) const {
    lp_hub_decide(tab, topo, gl, flt, v, pi[v], pp, gain, inx, sb, sc);
  }
};
struct RebHubPolicy {  // rebalancing selection
  static constexpr bool kWantBarrier = false;
  const int32_t* pi;
  const int32_t* vw;
  RebArgs a;
  GroupLayout gl;
  int32_t* dest;
  uint8_t* bkt;
  uint8_t* elig;
  const RefineState* st;
  __device__ bool run() const { return kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG)); }
  __device__ const Topo& topo_of() const { return a.topo; }
  __device__ int32_t topo_kc() const { return a.topo.kc; }
  __device__ int32_t words() const { return a.obj ? gl.total : a.topo.kc; }
  __device__ bool groups() const { return a.obj != 0; }
  __device__ bool want(int32_t v) const { return reb_eligible(a, pi[v], vw[v]); }
  __device__ void skip(int32_t v) const { elig[v] = 0; }
  __device__ void decide(const int32_t* tab, int32_t v, int32_t cv, int64_t* sb, int32_t* sc) const {
    reb_hub_decide(tab, a, a.topo.kc, gl, v, pi[v], cv, dest, bkt, elig, st, sb, sc);
  }
};

template <class P>
__global__ void __launch_bounds__(kHiThreads) k_hub_tab(GraphView g, HubRows hr, P pol, int64_t split_deg,
                                                        const int32_t* __restrict__ sidx, int32_t* gtab,
                                                        unsigned long long* ctr) {
  static_assert(kHiThreads == kSpanRows, "one thread per row of a span");
  extern __shared__ int32_t tab[];
  __shared__ int64_t sb[32];
  __shared__ int32_t sc[32];
  __shared__ int64_t s_ch;
  // the rows of the current span, checked at once
  __shared__ int32_t s_v[kSpanRows];  // the row's vertex; -1: nothing for this span to do
  __shared__ int64_t s_rb[kSpanRows], s_re[kSpanRows];
  __shared__ uint8_t s_split[kSpanRows];
  if (!pol.run()) return;
  const int32_t words = pol.words(), kc = pol.topo_kc();
  for (int32_t b = threadIdx.x; b < words; b += blockDim.x) tab[b] = 0;
  __syncthreads();
  const int64_t m_hub = hr.pre[hr.n_huge];
  const int64_t nspans = (hr.nchunks + kSpanChunks - 1) / kSpanChunks;
  for (int64_t sp = next_chunk(ctr, &s_ch); sp < nspans; sp = next_chunk(ctr, &s_ch)) {
    const int64_t cb = sp * kSpanChunks * kHubChunk, ce = min(cb + kSpanChunks * kHubChunk, m_hub);
    const int32_t r = hr.chunk[sp * kSpanChunks] + (int32_t)threadIdx.x;
    bool row = false;
    {
      int32_t v = -1;
      bool sp_row = false;
      int64_t rb = 0, re = 0;
      if (r < hr.n_huge) {
        rb = hr.pre[r];
        re = hr.pre[r + 1];
        row = rb < ce;
      }
      if (row) {
        sp_row = re - rb > split_deg;
        if (sp_row || rb >= cb) {  // a row up to split_deg is rated whole by the span of its first entry
          const int32_t u = hr.hi[hr.huge[r]];
          if (pol.want(u)) v = u;
          else if (!sp_row) pol.skip(u);  // (the finishing kernel skips the larger rows)
        }
      }
      s_v[threadIdx.x] = v;
      s_rb[threadIdx.x] = rb;
      s_re[threadIdx.x] = re;
      s_split[threadIdx.x] = sp_row;
    }
    const int nrows = __syncthreads_count(row);  // the span's rows are a prefix
    for (int i = 0; i < nrows; i++) {
      const int32_t v = s_v[i];
      if (v < 0) continue;
      const int64_t rb = s_rb[i], re = s_re[i];
      const int64_t x0 = g.xadj[v] - rb;
      if (!s_split[i]) {
        conn_add(g, x0 + rb, x0 + re, pol.pi, tab);
        __syncthreads();
        if (pol.groups()) conn_groups(pol.topo_of(), pol.gl, tab);
        pol.decide(tab, v, g.vw[v], sb, sc);
      } else {
        conn_add(g, x0 + max(rb, cb), x0 + min(re, ce), pol.pi, tab);
        __syncthreads();
        int32_t* G = gtab + (int64_t)sidx[hr.chunk[sp * kSpanChunks] + i] * kc;
        for (int32_t b = threadIdx.x; b < kc; b += blockDim.x)
          if (tab[b]) atomicAdd(&G[b], tab[b]);
        __syncthreads();
      }
      for (int32_t b = threadIdx.x; b < words; b += blockDim.x) tab[b] = 0;
      __syncthreads();
    }
  }
  leave_chunks(ctr);
}

// The larger rows, one CTA each (tickets): the summed table, then the decision.
template <class P>
__global__ void __launch_bounds__(kHiThreads) k_hub_tab_finish(GraphView g, HubRows hr, P pol,
                                                               const int32_t* __restrict__ split, int32_t n_split,
                                                               int32_t* gtab, unsigned long long* ctr) {
  extern __shared__ int32_t tab[];
  __shared__ int64_t sb[32];
  __shared__ int32_t sc[32];
  __shared__ int64_t s_j;
  if (!pol.run()) return;
  const int32_t words = pol.words(), kc = pol.topo_kc();
  for (int32_t b = threadIdx.x; b < words; b += blockDim.x) tab[b] = 0;
  __syncthreads();
  for (int64_t j = next_chunk(ctr, &s_j); j < n_split; j = next_chunk(ctr, &s_j)) {
    const int32_t v = hr.hi[hr.huge[split[j]]];
    const bool w = pol.want(v);
    if (P::kWantBarrier) __syncthreads();
    if (!w) {  // nothing was added to its table
      if (threadIdx.x == 0) pol.skip(v);
      continue;
    }
    int32_t* G = gtab + j * kc;
    for (int32_t b = threadIdx.x; b < kc; b += blockDim.x) {
      tab[b] = G[b];
      G[b] = 0;
    }
    __syncthreads();
    if (pol.groups()) conn_groups(pol.topo_of(), pol.gl, tab);
    pol.decide(tab, v, g.vw[v], sb, sc);
    for (int32_t b = threadIdx.x; b < words; b += blockDim.x) tab[b] = 0;
    __syncthreads();
  }
  leave_chunks(ctr);
}


// Compaction stores for the sort inputs.
struct LoadFlag2 {
  const uint8_t* a;
  const uint8_t* b;
  __device__ int64_t operator()(int64_t i) const { return (a[i] && b[i]) ? 1 : 0; }
};
struct StoreKeyed {
  const int32_t* keysrc;  // block code (pi) or destination
  const uint8_t* bkt;
  uint64_t* key;
  int32_t* val;
  __device__ void operator()(int64_t i, int64_t e, int64_t x) const {
    if (x) {
      key[e] = ((uint64_t)(uint32_t)keysrc[i] << kBucketBits) | bkt[i];
      val[e] = (int32_t)i;
    }
  }
};
struct LoadSortedWeight {
  const int32_t* val;
  const int32_t* vw;
  __device__ int64_t operator()(int64_t i) const { return vw[val[i]]; }
};
struct LoadRejected {
  const uint8_t* elig;
  const uint8_t* sel;
  const uint8_t* acc;
  const int32_t* vw;
  __device__ int64_t operator()(int64_t i) const { return (elig[i] && sel[i] && !acc[i]) ? vw[i] : 0; }
};
struct StoreIfPositive {
  int64_t* out;
  __device__ void operator()(int64_t i, int64_t e, int64_t x) const {
    if (x) out[i] = e;
  }
};

__global__ void k_copy_count(const int64_t* src, int64_t* dst) { *dst = *src; }

// Alg. 5 selection without sorting whole blocks.  In source block A the
// eligible vertices are ordered by (bucket, id) and v moves iff the weight
// before it is < E = c(A) - L_max.  With T_b the eligible weight of bucket b
// and C_b = T_0 + ... + T_{b-1}: buckets with C_b + T_b <= E move entirely,
// buckets with C_b >= E not at all, and in the one bucket with
// C_b < E < C_b + T_b a vertex moves iff the weight of the lower ids of that
// bucket is < rem = E - C_b.  Only that bucket needs an id order.
__global__ void __launch_bounds__(1024) k_reb_cut(const int64_t* __restrict__ W, int32_t kc, int64_t lmax,
                                                  int64_t* tab, int32_t* bcut, int64_t* rem, int64_t* cnt,
                                                  const RefineState* st) {
  if (!kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG))) return;
  for (int32_t A = threadIdx.x; A < kc; A += blockDim.x) {
    if (W[A] <= lmax) continue;  // only overloaded blocks have eligible vertices
    const int64_t E = W[A] - lmax;
    int64_t cum = 0, r = 0;
    int32_t cut = kBuckets;
    for (int b = 0; b < kBuckets; b++) {
      const int64_t t = tab[(int64_t)A * kBuckets + b];
      tab[(int64_t)A * kBuckets + b] = 0;  // the table is zero between steps
      if (cut == kBuckets) {
        if (cum + t <= E) {
          cum += t;
        } else {
          cut = b;
          r = E - cum;
        }
      }
    }
    bcut[A] = cut;
    rem[A] = r;
  }
  if (threadIdx.x == 0) cnt[CNT_ELIG] = 0;
}

// Buckets below the cut move, above it stay; the cut bucket's vertices go to
// a list keyed (block, id) whose order does not depend on the append order.
__global__ void k_reb_classify(int32_t n, const int32_t* __restrict__ pi, const uint8_t* __restrict__ elig,
                               const uint8_t* __restrict__ bkt, const int32_t* __restrict__ bcut,
                               const int64_t* __restrict__ rem, int idbits, uint8_t* sel, uint64_t* key,
                               int32_t* val, int64_t* cnt, const RefineState* st) {
  if (!kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG))) return;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!elig[v]) continue;
    const int32_t A = pi[v];
    const int32_t b = bkt[v], cut = bcut[A];
    if (b != cut) {
      sel[v] = b < cut ? 1 : 0;
      continue;
    }
    sel[v] = 0;
    if (rem[A] > 0) {
      const unsigned long long i = atomicAdd((unsigned long long*)&cnt[CNT_ELIG], 1ULL);
      key[i] = ((uint64_t)(uint32_t)A << idbits) | (uint64_t)v;
      val[i] = (int32_t)v;
    }
  }
}

// The cut-bucket list, when it has at most kSmallSort entries: one CTA sorts
// it by (block, id) in shared memory and selects by the per-block prefix.
__global__ void __launch_bounds__(kSmallThreads) k_reb_resolve(const uint64_t* __restrict__ kin,
                                                               const int32_t* __restrict__ vin,
                                                               const int64_t* __restrict__ cnt, int bits, int idbits,
                                                               const int32_t* __restrict__ vw,
                                                               const int64_t* __restrict__ rem, int64_t* headP,
                                                               uint8_t* sel, const RefineState* st,
                                                               cudaGraphConditionalHandle h_big, int use_h) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* ks = reinterpret_cast<uint64_t*>(smem_raw);
  int32_t* vs = reinterpret_cast<int32_t*>(ks + 2 * kSmallSort);
  int32_t* wcnt = vs + 2 * kSmallSort;
  __shared__ int32_t dbase[257];
  __shared__ int64_t sm[33];
  if (!kind_is(st, (1 << KIND_WEAK) | (1 << KIND_STRONG))) return;
  const int64_t n64 = cnt[CNT_ELIG];
  if (use_h && threadIdx.x == 0) cudaGraphSetConditional(h_big, n64 > kSmallSort ? 1u : 0u);
  if (n64 <= 0 || n64 > kSmallSort) return;
  const int n = (int)n64;
  for (int i = threadIdx.x; i < n; i += kSmallThreads) {
    ks[i] = kin[i];
    vs[i] = vin[i];
  }
  const int cur = cta_sort_small(ks, vs, wcnt, dbase, sm, n, bits);
  const uint64_t* k = ks + cur * kSmallSort;
  const int32_t* v = vs + cur * kSmallSort;
  constexpr int kItems = kSmallSort / kSmallThreads;
  const int first = threadIdx.x * kItems;
  int64_t c[kItems], local = 0;
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    c[j] = (first + j < n) ? vw[v[first + j]] : 0;
    local += c[j];
  }
  int64_t total;
  int64_t run = block_exclusive_scan(local, sm, &total);
  int64_t P[kItems];
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    P[j] = run;
    run += c[j];
    const int i = first + j;
    if (i < n && (i == 0 || (k[i] >> idbits) != (k[i - 1] >> idbits))) headP[k[i] >> idbits] = P[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kItems; j++) {
    const int i = first + j;
    if (i >= n) continue;
    const int32_t A = (int32_t)(k[i] >> idbits);
    sel[v[i]] = (P[j] - headP[A] < rem[A]) ? 1 : 0;
  }
}

// Larger cut-bucket lists: after a multi-CTA sort by (block, id).
__global__ void k_heads_shift(const uint64_t* __restrict__ key, const int64_t* __restrict__ P,
                              const int64_t* __restrict__ cnt, int shift, int64_t* headP) {
  const int64_t n = cnt[CNT_ELIG];
  if (n <= kSmallSort) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t grp = key[i] >> shift;
    if (i == 0 || (key[i - 1] >> shift) != grp) headP[grp] = P[i];
  }
}
__global__ void k_reb_mark_cut(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                               const int64_t* __restrict__ P, const int64_t* __restrict__ headP,
                               const int64_t* __restrict__ cnt, int shift, const int64_t* __restrict__ rem,
                               uint8_t* sel, unsigned long long* kcount, unsigned long long body) {
  const int64_t n = cnt[CNT_ELIG];
  if (kcount && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(kcount, body);
  if (n <= kSmallSort) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t A = (int32_t)(key[i] >> shift);
    sel[val[i]] = (P[i] - headP[A] < rem[A]) ? 1 : 0;
  }
}

__global__ void k_reb_apply_sel(int32_t n, const uint8_t* __restrict__ elig, const uint8_t* __restrict__ sel,
                                const int32_t* __restrict__ dest, int32_t* pi, const int32_t* __restrict__ vw,
                                int64_t* W, int32_t kc, RefineState* st) {
  __shared__ long long dW[kApplyCodes];
  if (st->kind != KIND_WEAK) return;
  BlockDelta bd{dW, W, kc <= kApplyCodes};
  bd.init(kc);
  __syncthreads();
  int32_t mine = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!elig[v] || !sel[v]) continue;
    const int32_t p = pi[v], q = dest[v];
    pi[v] = q;
    bd.move(p, q, vw[v]);
    mine++;
  }
  __syncthreads();
  bd.flush(kc);
  mine = warp_sum(mine);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&st->moved, mine);
}

// Segment heads of a sorted (group << 6 | bucket) list: headP[group] = P[i].
__global__ void k_heads(const uint64_t* __restrict__ key, const int64_t* __restrict__ P, const int64_t* d_n,
                        int64_t max_n, int64_t* headP) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n && i < max_n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t grp = key[i] >> kBucketBits;
    if (i == 0 || (key[i - 1] >> kBucketBits) != grp) headP[grp] = P[i];
  }
}

// strong: movers grouped by destination are accepted while it stays <= L_max
__global__ void k_reb_accept(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                             const int64_t* __restrict__ P, const int64_t* __restrict__ headP, const int64_t* d_n,
                             int64_t max_n, const int64_t* __restrict__ W, int64_t lmax,
                             const int32_t* __restrict__ vw, uint8_t* acc, int64_t* accepted) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n && i < max_n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = (int32_t)(key[i] >> kBucketBits);
    const int32_t v = val[i];
    const int64_t inc = P[i] + vw[v] - headP[d];
    const bool ok = W[d] + inc <= lmax;
    acc[v] = ok ? 1 : 0;
    if (ok) atomicAdd((unsigned long long*)&accepted[d], (unsigned long long)(int64_t)vw[v]);
  }
}

// residual room of the non-overloaded blocks in code order, prefix Rb
__global__ void __launch_bounds__(1024) k_reb_residual(const int64_t* __restrict__ W, const int64_t* __restrict__ accepted,
                                                       const int32_t* __restrict__ pe_of_code, int32_t kc,
                                                       int64_t lmax, int64_t* Rb) {
  __shared__ int64_t sm[33];
  int64_t carry = 0;
  for (int32_t base = 0; base < kc; base += blockDim.x) {
    const int32_t b = base + threadIdx.x;
    int64_t r = 0;
    if (b < kc && pe_of_code[b] >= 0 && W[b] <= lmax) {
      r = lmax - W[b] - accepted[b];
      if (r < 0) r = 0;
    }
    int64_t tot;
    const int64_t e = block_exclusive_scan(r, sm, &tot);
    if (b < kc) Rb[b] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) Rb[kc] = carry;
}

__global__ void k_reb_apply_strong(const uint64_t* __restrict__ key, const int32_t* __restrict__ val, const int64_t* d_n,
                                   int64_t max_n, const uint8_t* __restrict__ acc, const int64_t* __restrict__ sarr,
                                   const int64_t* __restrict__ Rb, int32_t kc, int32_t* pi,
                                   const int32_t* __restrict__ vw, int64_t* W, RefineState* st) {
  __shared__ long long dW[kApplyCodes];
  const int64_t n = *d_n;
  BlockDelta bd{dW, W, kc <= kApplyCodes};
  bd.init(kc);
  __syncthreads();
  int32_t mine = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n && i < max_n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = val[i];
    const int64_t c = vw[v];
    int32_t q = -1;
    if (acc[v]) {
      q = (int32_t)(key[i] >> kBucketBits);
    } else {
      // the room interval [Rb[b], Rb[b+1]) holding s: last b with Rb[b] <= s
      const int64_t s = sarr[v];
      int32_t lo = 0, hi = kc + 1;  // upper_bound over Rb[0..kc]
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (Rb[mid] <= s) lo = mid + 1;
        else hi = mid;
      }
      const int32_t b = lo - 1;
      if (b >= 0 && b < kc && s + c <= Rb[b + 1]) q = b;
    }
    if (q < 0) continue;
    const int32_t p = pi[v];
    pi[v] = q;
    bd.move(p, q, c);
    mine++;
  }
  __syncthreads();
  bd.flush(kc);
  mine = warp_sum(mine);  // one update of the shared counter per warp
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&st->moved, mine);
}

// ---------------------------------------------------------------------------
// Alg. 6 controller (one CTA): best-state tracking, patience, next step kind
// ---------------------------------------------------------------------------


// Maximum block weight over the code space (all threads of the block call
// it; thread 0 gets the result).
__device__ __forceinline__ int64_t block_max_w(const int64_t* __restrict__ W, int32_t kc, int64_t* smax) {
  int64_t mx = 0;
  for (int32_t b = threadIdx.x; b < kc; b += blockDim.x) mx = W[b] > mx ? W[b] : mx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = smax[w] > mx ? smax[w] : mx;
  return mx;
}

// One Alg. 6 decision (thread 0): the best-mapping and patience updates on
// J and the maximum block weight of P' after a move, and the kind of the next
// step.
__device__ void control_step(RefineState* s, int64_t mx, int64_t J, const CtlArgs& a, int phase,
                             cudaGraphConditionalHandle h_loop, int use_handle) {
  if (phase == 1 && s->done) {
    if (use_handle) cudaGraphSetConditional(h_loop, 0u);
    return;
  }
  s->copy_best = 0;
  s->J = J;
  s->maxw = mx;
  s->last_kind = s->kind;
  if (phase == 0) {
    s->best_J = J;
    s->best_maxw = mx;
    s->i = 0;
    s->iw = 0;
    s->t = 0;
    s->done = 0;
  } else {
    const int32_t t = s->t;
    if (t - 1 < a.tcap) {
      a.tk[t - 1] = s->kind;
      a.tJ[t - 1] = J;
      a.tW[t - 1] = mx;
    }
    if (mx <= a.lmax) {
      if (s->best_maxw > a.lmax) {  // a feasible mapping replaces an infeasible best
        s->best_J = J;
        s->best_maxw = mx;
        s->copy_best = 1;
        s->i = 0;
      } else {
        // both tests compare with the best J before it is replaced
        const bool reset = (__int128)a.phi_den * J < (__int128)a.phi_num * s->best_J;
        if (J < s->best_J) {
          s->best_J = J;
          s->best_maxw = mx;
          s->copy_best = 1;
        }
        if (reset) s->i = 0;
      }
    } else if (mx < s->best_maxw) {
      s->best_J = J;
      s->best_maxw = mx;
      s->copy_best = 1;
      s->i = 0;
    }
  }
  // Alg. 6 terminates (each patience reset needs a 0.1 % better J or a lower
  // maximum block weight); the cap on t only bounds the loop by construction
  // and also keeps t inside the 20 bits of the rebalancing hash.
  const bool capped = s->t >= kMaxRefineIters;
  if (capped && s->rounds < 0) s->capped = 1;
  const bool stop = capped || (s->rounds >= 0 ? (s->t >= s->rounds) : (s->i >= a.patience));
  s->moved = 0;
  if (use_handle) cudaGraphSetConditional(h_loop, stop ? 0u : 1u);
  if (stop) {
    s->done = 1;
    s->kind = KIND_NONE;
    return;
  }
  s->i++;
  s->t++;
  if (mx <= a.lmax) {
    s->kind = KIND_LP;
    s->iw = 0;
  } else if (s->iw < a.weak_max) {
    s->kind = KIND_WEAK;
    s->iw++;
  } else {
    s->kind = KIND_STRONG;
    s->iw = 0;
  }
}

// Value of the J accumulator for the step just decided: the current J when
// that step adds its exact change (LP, weak), else 0 (a full evaluation).
__device__ __forceinline__ int64_t next_j_base(const RefineState* s, int64_t J) {
  return (s->kind == KIND_LP || s->kind == KIND_WEAK) ? J : 0;
}

// Every block of a J evaluation arrives here once its part of J is in the
// accumulator; the last one to arrive takes the Alg. 6 decision on the
// complete J (all blocks have read the step kind by then).
__device__ void eval_finish(int64_t* Jacc, const EvalCtl& ec) {
  __shared__ unsigned int last;
  __shared__ int64_t smax[32];
  if (!ec.s) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ec.ctr, 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int64_t mx = block_max_w(ec.W, ec.a.kc, smax);
  if (threadIdx.x == 0) {
    const int64_t J = (int64_t)atomicAdd((unsigned long long*)Jacc, 0ULL);
    *ec.ctr = 0;
    control_step(ec.s, mx, J, ec.a, ec.phase, ec.h, ec.use_h);
    *Jacc = next_j_base(ec.s, J);
  }
}



// Kernels run by one graph iteration: the fixed nodes plus the body of the
// step that ran (the kind is recorded by k_control before it moves on).
struct IterCounts {
  unsigned long long fixed, lp, reb, strong;
};

__global__ void k_state_init(RefineState* s, int32_t rounds, int32_t level) {
  RefineState z{};
  z.rounds = rounds;
  z.level = level;
  *s = z;
}

__global__ void k_copy_best(RefineState* s, const int32_t* __restrict__ pi, int32_t* __restrict__ best, int32_t n,
                            IterCounts ic) {
  if (ic.fixed && blockIdx.x == 0 && threadIdx.x == 0) {
    const int32_t k = s->last_kind;
    s->kernels += ic.fixed + (k == KIND_LP ? ic.lp : 0) + ((k == KIND_WEAK || k == KIND_STRONG) ? ic.reb : 0) +
                  (k == KIND_STRONG ? ic.strong : 0);
  }
  if (!s->copy_best) return;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    best[v] = pi[v];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline unsigned grid_for(const Ctx& c, int64_t items_per_block, int64_t n) {
  int64_t g = (n + items_per_block - 1) / items_per_block;
  int64_t cap = (int64_t)c.num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

size_t conn_smem(const Ctx& c) { return (size_t)group_layout(c.topo).total * sizeof(int32_t); }

// Grid of a mid-degree kernel (one warp per vertex of the high-degree list).
inline unsigned mid_grid(Ctx& c, const void* fn, size_t smem, int64_t n_hi) {
  int64_t g = (n_hi + kMidWarps - 1) / kMidWarps;
  const int64_t cap = (int64_t)c.num_sms * c.resident_blocks(fn, kMidThreads, smem);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// The dense per-warp tables of the mid-degree LP gain and rebalancing kernels
// fit in shared memory (else the CTA-per-vertex kernels take every vertex of
// degree > kLowDeg).
inline bool mid_tables(const Ctx& c) { return group_layout(c.topo).total <= kMidTableMax; }
inline size_t mid_table_smem(int32_t words) { return (size_t)kMidWarps * words * sizeof(int32_t); }

// The two launches of a hub table kernel (the second only for rows summed
// over chunks), each one wave of resident CTAs drawing tickets.
template <class P>
void launch_hub_tab(Ctx& c, Level& L, const P& pol, size_t smem) {
  const void* f1 = (const void*)k_hub_tab<P>;
  const int64_t r1 = (int64_t)c.num_sms * c.resident_blocks(f1, kHiThreads, smem);
  const int64_t spans = (L.n_hub_chunks + kSpanChunks - 1) / kSpanChunks;
  k_hub_tab<P><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(spans, r1)), kHiThreads, smem, c.st>>>(
      view(L), hub_rows(L), pol, L.hub_split_deg, L.hub_sidx, L.hub_gtab, c.hub_ctr);
  count_launch();
  if (L.n_split) {
    const void* f2 = (const void*)k_hub_tab_finish<P>;
    const int64_t r2 = (int64_t)c.num_sms * c.resident_blocks(f2, kHiThreads, smem);
    k_hub_tab_finish<P><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(L.n_split, r2)), kHiThreads, smem, c.st>>>(
        view(L), hub_rows(L), pol, L.hub_split, L.n_split, L.hub_gtab, c.hub_ctr);
    count_launch();
  }
}

// J of the current mapping of a level; with `ec`, the last block of the
// low-degree pass also takes the Alg. 6 decision (the high-degree pass runs
// first so that J is complete then).
// full: the launch streams the whole CSR (false when it only closes an LP or
// weak step whose exact change of J is already accumulated)
void launch_eval(Ctx& c, int lvl, const EvalCtl* ec = nullptr, bool full = true) {
  Level& L = c.lv[lvl];
  c.prof_level = lvl;
  cudaEvent_t ev = nullptr;
  // per vertex xadj (8) + P(v) (4), per entry adjacency (4) + weight (4) + P(u) (4), per degree class
  if (L.n_hi > L.n_huge) {
    if (full) ev = c.prof_begin();
    k_eval_mid<<<mid_grid(c, (const void*)k_eval_mid, 0, L.n_hi), kMidThreads, 0, c.st>>>(
        view(L), L.hi, L.n_hi, L.pi, c.topo, c.Jacc, ec ? ec->s : nullptr, ec ? ec->phase : 0); count_launch();
    if (full) c.prof_end(ev, PK_EVAL_MID, 12 * (int64_t)(L.n_hi - L.n_huge) + 12 * (L.m_hi - L.m_huge));
  }
  if (L.n_huge) {
    if (full) ev = c.prof_begin();
    k_eval_high<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(L.n_hub_chunks, (int64_t)c.num_sms * 8)), kHiThreads,
                  0, c.st>>>(view(L), hub_rows(L), L.pi, c.topo, c.Jacc, ec ? ec->s : nullptr, ec ? ec->phase : 0);
    count_launch();
    if (full) c.prof_end(ev, PK_EVAL_HIGH, 12 * (int64_t)L.n_huge + 12 * L.m_huge);
  }
  ev = c.prof_begin();
  const EvalCtl none{nullptr, nullptr, nullptr, CtlArgs{}, 0, 0, 0};
  k_eval_tile<<<tile_grid(c, (const void*)k_eval_tile, L.n), kTileThreads, 0, c.st>>>(view(L), L.pi, c.topo, c.Jacc,
                                                                                       ec ? *ec : none); count_launch();
  // xadj (8) + P(v) (4) per vertex; adjacency (4) + weight (4) + gathered P(u) (4) per entry
  if (full) c.prof_end(ev, PK_EVAL, 12 * (int64_t)(L.n - L.n_hi) + 12 * (L.m - L.m_hi));
  else c.prof_end(ev, PK_EVAL_CTL, 0);
}

template <class Mv>
void launch_delta(Ctx& c, int lvl, Mv mv, int kind) {
  Level& L = c.lv[lvl];
  k_delta_low<Mv><<<grid_for(c, kThreads / kSubWarp, L.n), kThreads, 0, c.st>>>(view(L), L.pi, mv, c.topo, c.Jacc,
                                                                                 c.state, kind); count_launch();
  if (L.n_hi > L.n_huge) {
    k_delta_mid<Mv><<<mid_grid(c, (const void*)k_delta_mid<Mv>, 0, L.n_hi), kMidThreads, 0, c.st>>>(
        view(L), L.hi, L.n_hi, L.pi, mv, c.topo, c.Jacc, c.state, kind); count_launch();
  }
  if (L.n_huge)
    k_delta_high<Mv><<<(unsigned)std::max<int64_t>(
                           1, std::min<int64_t>((L.n_hub_chunks + kSpanChunks - 1) / kSpanChunks, (int64_t)c.num_sms * 8)),
                       kHiThreads, 0, c.st>>>(view(L), hub_rows(L), L.pi, mv, c.topo, c.Jacc, c.state, kind);
  if (L.n_huge) count_launch();
}

void launch_lp(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  const unsigned gl = grid_for(c, kThreads / kSubWarp, L.n);
  const bool mid_tab = mid_tables(c);
  const GroupLayout glay = group_layout(c.topo);
  // vertices of degree > kLowDeg left to the CTA-per-vertex kernels
  const int32_t* gsel = mid_tab ? L.huge : nullptr;
  const int32_t ng = mid_tab ? L.n_huge : L.n_hi;
  c.prof_level = lvl;
  cudaEvent_t ev = c.prof_begin();
  const LpFilter flt{c.cfg.lp_relax_num, c.cfg.lp_relax_den};
  k_lp_gain_tile<<<tile_grid(c, (const void*)k_lp_gain_tile, L.n), kTileThreads, 0, c.st>>>(view(L), L.pi, c.lock, c.pp, c.gain, c.inx, c.topo,
                                                                flt, c.state); count_launch();
  // per vertex: xadj 8, P 4, lock 1, X 1, P' 4, g 8; per entry: adjacency 4, weight 4, gathered P(u) 4
  c.prof_end(ev, PK_LP_GAIN, 26 * (int64_t)(L.n - L.n_hi) + 12 * (L.m - L.m_hi));
  if (mid_tab && L.n_hi > L.n_huge) {
    const size_t sm = mid_table_smem(glay.total);
    ev = c.prof_begin();
    k_lp_gain_mid<<<mid_grid(c, (const void*)k_lp_gain_mid, sm, L.n_hi), kMidThreads, sm, c.st>>>(
        view(L), L.hi, L.n_hi, L.pi, c.lock, c.pp, c.gain, c.inx, c.topo, glay, flt, c.state); count_launch();
    c.prof_end(ev, PK_LP_GAIN_MID, 26 * (int64_t)(L.n_hi - L.n_huge) + 12 * (L.m_hi - L.m_huge));
  }
  if (ng) {
    const int64_t me = mid_tab ? L.m_huge : L.m_hi;
    ev = c.prof_begin();
    if (mid_tab) {
      const LpHubPolicy pol{L.pi, c.lock, c.pp, c.gain, c.inx, c.topo, glay, flt, c.state};
      launch_hub_tab(c, L, pol, (size_t)glay.total * sizeof(int32_t));
    } else {
      k_lp_gain_high<<<std::max(1, std::min(ng, c.num_sms * 8)), kHiThreads, conn_smem(c), c.st>>>(
          view(L), L.hi, gsel, ng, L.pi, c.lock, c.pp, c.gain, c.inx, c.topo, glay, flt, c.state); count_launch();
    }
    c.prof_end(ev, PK_LP_GAIN_HIGH, 26 * (int64_t)ng + 12 * me);
  }
  ev = c.prof_begin();
  k_lp_after_low<<<gl, kThreads, 0, c.st>>>(view(L), L.pi, c.pp, c.gain, c.inx, c.lock, c.topo, c.state); count_launch();
  // the X flag of every vertex (the work on X itself is data dependent)
  c.prof_end(ev, PK_LP_AFTER, (int64_t)(L.n - L.n_hi));
  if (L.n_hi > L.n_huge) {
    k_lp_after_mid<<<mid_grid(c, (const void*)k_lp_after_mid, 0, L.n_hi), kMidThreads, 0, c.st>>>(
        view(L), L.hi, L.n_hi, L.pi, c.pp, c.gain, c.inx, c.lock, c.topo, c.state); count_launch();
  }
  if (L.n_huge) {
    const int64_t res = (int64_t)c.num_sms * c.resident_blocks((const void*)k_lp_after_hub, kHiThreads, 0);
    const int64_t spans = (L.n_hub_chunks + kSpanChunks - 1) / kSpanChunks;
    k_lp_after_hub<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(spans, res)), kHiThreads, 0, c.st>>>(
        view(L), hub_rows(L), L.pi, c.pp, c.gain, c.inx, L.hub_acc, c.topo, c.state, c.hub_ctr);
    count_launch();
    k_lp_after_hub_finish<<<grid_for(c, kThreads, L.n_huge), kThreads, 0, c.st>>>(hub_rows(L), c.inx, L.hub_acc,
                                                                                c.lock, c.state);
    count_launch();
  }
  launch_delta(c, lvl, LpMoves{c.lock, c.pp}, KIND_LP);
  k_lp_apply<<<grid_for(c, kThreads, L.n), kThreads, 0, c.st>>>(L.n, L.pi, c.pp, c.lock, L.vw, c.W, c.topo.kc,
                                                                 c.state); count_launch();
}

RebPrepArgs reb_prep_args(const Ctx& c) {
  return RebPrepArgs{c.W, c.d_pe_of_code, c.topo, c.lmax, c.cV, c.cfg.sigma_gap, c.U, c.counters, c.accepted};
}

void launch_rebalance(Ctx& c, int lvl, bool prep_done = false) {
  Level& L = c.lv[lvl];
  const int64_t n = L.n;
  uint8_t* bucket = c.sel;    // loss bucket per eligible vertex
  uint8_t* selected = c.inx;  // selection flag per eligible vertex (X is free while rebalancing)
  if (!prep_done) {
    k_reb_prep<<<1, 1024, 0, c.st>>>(reb_prep_args(c), c.state); count_launch();
  }
  RebArgs a{c.W, c.U, c.counters, c.tab, c.lmax, c.cV, c.k, c.cfg.seed, c.cfg.reb_objective, c.topo};
  k_reb_select_low<<<grid_for(c, kThreads / kSubWarp, n), kThreads, 0, c.st>>>(view(L), L.pi, a, c.dest, bucket,
                                                                                 c.elig, c.state); count_launch();
  if (L.n_hi) {
    const GroupLayout gl = group_layout(c.topo);
    const int32_t words = c.cfg.reb_objective ? gl.total : c.topo.kc;
    const size_t smem = (size_t)words * sizeof(int32_t);
    const bool mid_tab = mid_tables(c);
    if (mid_tab && L.n_hi > L.n_huge) {
      const size_t sm = mid_table_smem(words);
      k_reb_select_mid<<<mid_grid(c, (const void*)k_reb_select_mid, sm, L.n_hi), kMidThreads, sm, c.st>>>(
          view(L), L.hi, L.n_hi, L.pi, a, c.topo.kc, gl, c.dest, bucket, c.elig, c.state); count_launch();
    }
    const int32_t ng = mid_tab ? L.n_huge : L.n_hi;
    if (ng && mid_tab) {
      const RebHubPolicy pol{L.pi, L.vw, a, gl, c.dest, bucket, c.elig, c.state};
      launch_hub_tab(c, L, pol, smem);
    } else if (ng) {
      k_reb_select_high<<<std::max(1, std::min(ng, c.num_sms * 8)), kHiThreads, smem, c.st>>>(
          view(L), L.hi, nullptr, ng, L.pi, a, c.topo.kc, gl, c.dest, bucket, c.elig, c.state);
      count_launch();
    }
  }
  k_reb_cut<<<1, 1024, 0, c.st>>>(c.W, c.topo.kc, c.lmax, c.tab, c.bcut, c.rem, c.counters, c.state); count_launch();
  const int idbits = bits_for_n(n);
  const int bits = c.topo.code_bits + idbits;
  const unsigned g = grid_for(c, kThreads, n);
  k_reb_classify<<<g, kThreads, 0, c.st>>>(L.n, L.pi, c.elig, bucket, c.bcut, c.rem, idbits, selected, c.sort.key[0],
                                           c.sort.val[0], c.counters, c.state); count_launch();
  cudaGraphConditionalHandle h = c.cap.on() ? cap_handle(c.st, 0) : 0;
  k_reb_resolve<<<1, kSmallThreads, small_sort_smem(), c.st>>>(c.sort.key[0], c.sort.val[0], c.counters, bits, idbits,
                                                               L.vw, c.rem, c.headP, selected, c.state, h,
                                                               c.cap.on() ? 1 : 0); count_launch();
  int64_t* d_list = c.counters + CNT_ELIG;
  auto big = [&](cudaStream_t bs, unsigned long long* kcount, long long* body) {
    cudaStream_t saved = c.st;
    c.st = bs;
    const int cur = radix_sort_pairs(c.sort, n, d_list, bits, bs);
    scan(LoadSortedWeight{c.sort.val[cur], L.vw}, StoreExcl{c.P64}, n, d_list, c.scan, bs);
    k_heads_shift<<<g, kThreads, 0, bs>>>(c.sort.key[cur], c.P64, c.counters, idbits, c.headP); count_launch();
    const unsigned long long bk = body ? (unsigned long long)(*body + 1) : 0ULL;
    k_reb_mark_cut<<<g, kThreads, 0, bs>>>(c.sort.key[cur], c.sort.val[cur], c.P64, c.headP, c.counters, idbits, c.rem,
                                          selected, kcount, bk); count_launch();
    c.st = saved;
  };
  if (c.cap.on()) {
    long long body = 0;
    long long* outer = set_capture_counter(&body);
    cap_cond(c.cap, c.st, h, cudaGraphCondTypeIf, [&](cudaStream_t bs) { big(bs, &c.state->kernels, &body); });
    set_capture_counter(outer);
  } else {
    big(c.st, nullptr, nullptr);
  }
  launch_delta(c, lvl, WeakMoves{c.elig, selected, c.dest}, KIND_WEAK);
  k_reb_apply_sel<<<g, kThreads, 0, c.st>>>(L.n, c.elig, selected, c.dest, L.pi, L.vw, c.W, c.topo.kc, c.state);
  count_launch();
}

__global__ void k_strong_gate(const RefineState* st, int64_t* d_sel) {
  if (st->kind != KIND_STRONG) *d_sel = 0;
}

// ---------------------------------------------------------------------------
// Fused engine: the whole Alg. 6 run of one small level (or of every graph
// of a batch, one cluster each) in a single launch of thread-block clusters.
// The phases of an iteration are separated by cluster barriers instead of
// kernel boundaries; rows of at most kEngLaneDeg entries are taken by warp
// tiles (one lane or an 8-lane sub-warp per vertex), larger rows by whole
// CTAs (dense connectivity tables over the PE codes in shared memory, as the
// hub kernels of the stream path); the serial steps (sorts, cut, strong
// tail, the controller) run in the cluster's first CTA.  Arrays written
// inside the launch are read through plain pointers (no read-only path), and
// the barriers order the phases across the cluster's SMs.
// ---------------------------------------------------------------------------
constexpr int kEngThreads = 1024;
constexpr int kEngMaxN = 1 << 15;   // default: levels of at most this many vertices use the engine
constexpr int kEngLaneDeg = 128;    // larger rows are taken by whole CTAs
constexpr int kEngMaxCluster = 16;
static_assert(kEngThreads == kSmallThreads, "the engine's CTA sorts with the single-CTA sort");

struct EngineJob {
  GraphView g;
  int32_t* pi;
  int32_t* pp;
  int64_t* gain;
  uint8_t* inx;
  uint8_t* lock;
  int32_t* best;
  int32_t* dest;
  uint8_t* elig;
  uint8_t* bkt;
  uint8_t* sel;
  uint8_t* acc;
  int64_t* sarr;
  int64_t* P;  // [n + 1]
  int64_t* W;
  int64_t* accepted;
  int32_t* U;
  int64_t* tab;
  int32_t* bcut;
  int64_t* rem;
  int64_t* headP;
  int64_t* Rb;
  uint64_t* key0;
  int32_t* val0;
  uint64_t* key1;
  int32_t* val1;
  int64_t* cnt;
  int64_t* Jacc;
  RefineState* s;
  const int32_t* pe_of_code;
  Topo topo;
  CtlArgs ctl;
  int64_t lmax;
  int64_t cV;
  uint64_t seed;
  int32_t k;
  int32_t sigma_gap;
  int32_t level;
  int32_t rounds;
  LpFilter flt;
  int32_t reb_obj;  // rebalancing gains: 0 cut, 1 Eq. 1
  // rows of degree > kEngLaneDeg: found among the vertices of degree > kLowDeg
  const int32_t* hi;
  int32_t n_hi;
  int32_t has_heavy;  // some row has more than kEngLaneDeg entries
  GroupLayout gl;     // connectivity table layout of those rows
};

struct PlainRow {  // neighbour PEs through plain loads (the mapping changes inside the launch)
  const int32_t* __restrict__ adj;
  const int32_t* __restrict__ adjw;
  const int32_t* pi;
  __device__ __forceinline__ int32_t code(int j) const { return pi[adj[j]]; }
  __device__ __forceinline__ int32_t weight(int j) const { return adjw[j]; }
};

// Barrier between the engine's phases: the cluster's hardware barrier, or a
// grid-wide barrier for the cooperative launch over all SMs.
struct ClusterSync {
  __device__ __forceinline__ void sync() const { cg::this_cluster().sync(); }
};

// Grid barrier state (zero-initialised; count returns to 0 after each use).
struct GridBar {
  unsigned int count;
  unsigned int gen;
  unsigned int err;  // set when a wait gave up
  unsigned int pad;
};
constexpr unsigned long long kBarWaitNs = 1000000000ULL;  // a wait gives up after one second
constexpr unsigned kBarSpinLimit = 1u << 26;               // and after this many polls in any case

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct GridSync {
  GridBar* bar;
  unsigned int* flag;  // shared memory of the calling block
  unsigned int need;   // arrivals that release the barrier (gridDim.x)
  // Every block arrives once; the last one resets the count and advances the
  // generation the others poll.  Fences order each block's phase writes
  // before its arrival and the following reads after the release.  A wait
  // that exceeds the limit marks the barrier failed; the blocks then leave
  // the kernel at their next barrier and the host reports the failure.
  __device__ __forceinline__ void sync() const {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned g0 = *(volatile unsigned*)&bar->gen;
      __threadfence();
      if (atomicAdd(&bar->count, 1u) == need - 1) {
        bar->count = 0;
        __threadfence();
        atomicAdd(&bar->gen, 1u);
      } else {
        unsigned spins = 0;
        const unsigned long long t0 = global_ns();
        while (*(volatile unsigned*)&bar->gen == g0) {
          if (++spins > kBarSpinLimit || global_ns() - t0 > kBarWaitNs || *(volatile unsigned*)&bar->err) {
            atomicOr(&bar->err, 1u);
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
      *flag = *(volatile unsigned*)&bar->err;
    }
    __syncthreads();
    if (*(volatile unsigned*)flag) asm volatile("exit;");
  }
};

__device__ __forceinline__ void eng_sync() { cg::this_cluster().sync(); }

// block-wide exclusive scan over chunks of blockDim values: f(i) for i < n,
// out(i, exclusive, value); returns the total (all threads)
template <class F, class O>
__device__ int64_t cta_scan(int64_t n, F f, O out, int64_t* sm) {
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t x = i < n ? f(i) : 0;
    int64_t tot;
    const int64_t e = block_exclusive_scan(x, sm, &tot);
    if (i < n) out(i, carry + e, x);
    carry += tot;
  }
  return carry;
}

struct EngSmem {
  int32_t hist[256];
  int32_t ctot[256];
  int32_t dbase[256];
  int32_t wcnt[32 * 256];
  int64_t sm[33];
  int32_t sdist[32];
  int64_t smax[32];
  int64_t hb[32];  // per-warp best scores of a CTA-wide row decision
  int32_t hc[32];  // and their codes
};

// Stable LSD radix sort (8-bit digits) of n pairs by one CTA through global
// buffers: per pass a digit histogram, then chunks of blockDim elements in
// index order, ranked within the chunk by warp matching.  Returns 0 or 1,
// the buffer holding the result.
__device__ int cta_sort_global(uint64_t* k0, int32_t* v0, uint64_t* k1, int32_t* v1, int n, int bits, EngSmem& S) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const unsigned lt = (1u << l) - 1u;
  const int nw = blockDim.x >> 5;
  uint64_t* K[2] = {k0, k1};
  int32_t* V[2] = {v0, v1};
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    for (int d = threadIdx.x; d < 256; d += blockDim.x) S.hist[d] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&S.hist[(int)((K[cur][i] >> shift) & 255u)], 1);
    __syncthreads();
    {
      const int64_t x = threadIdx.x < 256 ? S.hist[threadIdx.x] : 0;
      int64_t tot;
      const int64_t e = block_exclusive_scan(x, S.sm, &tot);
      if (threadIdx.x < 256) S.hist[threadIdx.x] = (int32_t)e;  // running offset of each digit
    }
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
      for (int i = threadIdx.x; i < nw * 256; i += blockDim.x) S.wcnt[i] = 0;
      __syncthreads();
      const int i = base + threadIdx.x;
      const bool valid = i < n;
      const uint64_t key = valid ? K[cur][i] : 0;
      const int32_t val = valid ? V[cur][i] : 0;
      const int d = valid ? (int)((key >> shift) & 255u) : 256 + l;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int r = __popc(peers & lt);
      if (valid && (peers & lt) == 0) S.wcnt[w * 256 + d] = __popc(peers);
      __syncthreads();
      if (threadIdx.x < 256) {
        int32_t run = 0;
        for (int ww = 0; ww < nw; ww++) {
          const int32_t t = S.wcnt[ww * 256 + threadIdx.x];
          S.wcnt[ww * 256 + threadIdx.x] = run;
          run += t;
        }
        S.ctot[threadIdx.x] = run;
      }
      __syncthreads();
      if (valid) {
        const int pos = S.hist[d] + S.wcnt[w * 256 + d] + r;
        K[cur ^ 1][pos] = key;
        V[cur ^ 1][pos] = val;
      }
      __syncthreads();
      if (threadIdx.x < 256) S.hist[threadIdx.x] += S.ctot[threadIdx.x];
      __syncthreads();
    }
    cur ^= 1;
  }
  return cur;
}

// Sorts the n (key, value) pairs in J.key0 / J.val0 by key bits [0, bits)
// (stable), by the calling CTA: in shared memory (dyn) when n <= kSmallSort,
// else through the global double buffers.  K / V point to the result.
__device__ void eng_sort(const EngineJob& J, EngSmem& S, int32_t* dyn, int n, int bits, const uint64_t*& K,
                         const int32_t*& V) {
  if (n <= (int)blockDim.x) {
    // rank sort: the position of pair i is the number of pairs with a smaller
    // key, or an equal key and a smaller index (stable)
    uint64_t* ks = reinterpret_cast<uint64_t*>(dyn);
    int32_t* vs = reinterpret_cast<int32_t*>(ks + 2 * kSmallSort);
    const uint64_t mask = bits >= 64 ? ~0ULL : ((1ULL << bits) - 1ULL);
    const int i = threadIdx.x;
    uint64_t ki = 0;
    int32_t vi = 0;
    if (i < n) {
      ki = J.key0[i] & mask;
      vi = J.val0[i];
      ks[i] = ki;
    }
    __syncthreads();
    if (i < n) {
      int r = 0;
      for (int j = 0; j < n; j++) {
        const uint64_t kj = ks[j];
        r += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
      }
      ks[kSmallSort + r] = J.key0[i];
      vs[kSmallSort + r] = vi;
    }
    __syncthreads();
    K = ks + kSmallSort;
    V = vs + kSmallSort;
  } else if (n <= kSmallSort) {
    uint64_t* ks = reinterpret_cast<uint64_t*>(dyn);
    int32_t* vs = reinterpret_cast<int32_t*>(ks + 2 * kSmallSort);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      ks[i] = J.key0[i];
      vs[i] = J.val0[i];
    }
    __syncthreads();
    const int cur = cta_sort_small(ks, vs, S.wcnt, S.dbase, S.sm, n, bits);
    K = ks + cur * kSmallSort;
    V = vs + cur * kSmallSort;
  } else {
    const int cur = cta_sort_global(J.key0, J.val0, J.key1, J.val1, n, bits, S);
    K = cur ? J.key1 : J.key0;
    V = cur ? J.val1 : J.val0;
  }
}

// Alg. 5 destination of one vertex (thread level): edge-cut gain, lowest id
// on ties, the random-block fallback; returns false if the vertex cannot move.
template <bool kJ>
__device__ bool eng_reb_select(const EngineJob& J, int32_t v, int64_t sigma, int64_t nU, int32_t t,
                               const int32_t* sdist, int32_t& dst, int32_t& bucket) {
  const GraphView& g = J.g;
  const int32_t A = J.pi[v];
  const int64_t WA = J.W[A];
  if (WA <= J.lmax) return false;
  if (2 * (int64_t)J.k * g.vw[v] > 3 * ((int64_t)J.k * WA - J.cV)) return false;
  const int64_t b = g.xadj[v], e = g.xadj[v + 1];
  const PlainRow row{g.adj + b, g.adjw + b, J.pi};
  const int deg = (int)(e - b);
  // score: conn(v, q), or -T(q) for the J gains (kJ)
  using Score = typename std::conditional<kJ, int64_t, int32_t>::type;
  Score connA = 0, bconn = 0;
  if constexpr (kJ) connA = -row_cost(row, deg, sdist, A);
  int32_t bc = INT32_MAX;
  bool found = false;
  for (int64_t x = b; x < e; x++) {
    const int32_t c = J.pi[g.adj[x]];
    if (c == A) {
      if constexpr (!kJ) connA += g.adjw[x];
      continue;
    }
    if (J.W[c] > sigma) continue;
    bool seen = false;
    for (int64_t y = b; y < x; y++)
      if (J.pi[g.adj[y]] == c) {
        seen = true;
        break;
      }
    if (seen) continue;
    Score cc = 0;
    if constexpr (kJ) {
      cc = -row_cost(row, deg, sdist, c);
    } else {
      for (int64_t y = x; y < e; y++) cc += (J.pi[g.adj[y]] == c) ? g.adjw[y] : 0;
    }
    if (!found || cc > bconn || (cc == bconn && c < bc)) {
      bconn = cc;
      bc = c;
      found = true;
    }
  }
  int64_t gcut;
  if (found) {
    gcut = (int64_t)bconn - connA;
  } else if (nU > 0) {
    bc = J.U[h_rebalance(J.seed, J.level, t, v) % (uint64_t)nU];
    int64_t sr = 0;  // the drawn block is not a neighbour
    if constexpr (kJ) sr = -row_cost(row, deg, sdist, bc);
    gcut = sr - connA;
  } else {
    return false;
  }
  dst = bc;
  bucket = loss_bucket(gcut);
  return true;
}

// Cluster-wide position of the calling thread.
struct EngGeom {
  int64_t gt, GT;  // thread index and thread count of the cluster
  int64_t gw, GW;  // warp index and warp count of the cluster
  int cta, ncta;   // CTA index and CTA count of the cluster
  int lane;
  bool lead;  // first CTA of the cluster
};

// Whether a row of `deg` entries is taken by a whole CTA.
__device__ __forceinline__ bool eng_heavy(const EngineJob& J, int64_t deg) {
  return J.has_heavy && deg > kEngLaneDeg;
}
// The same for vertex v (its row bounds are read only when the level has such rows).
__device__ __forceinline__ bool eng_heavy_row(const EngineJob& J, int64_t v) {
  return J.has_heavy && J.g.xadj[v + 1] - J.g.xadj[v] > kEngLaneDeg;
}

// Calls f(v, b, e) for every row of more than kEngLaneDeg entries that falls
// to the calling CTA (rows dealt round-robin over the cluster's CTAs); all
// threads of the CTA take the same rows.
template <class F>
__device__ __forceinline__ void eng_heavy_rows(const EngineJob& J, const EngGeom& eg, F f) {
  if (!J.has_heavy) return;
  for (int32_t h = eg.cta; h < J.n_hi; h += eg.ncta) {
    const int32_t v = J.hi[h];
    const int64_t b = J.g.xadj[v], e = J.g.xadj[v + 1];
    if (e - b > kEngLaneDeg) f(v, b, e);
  }
}

// Dense connectivity table of one row in shared memory (`total` entries
// zeroed first): conn per PE code, and with `groups` the level group sums
// (the layout of GroupLayout).  The mapping is read through plain loads.
// All threads of the CTA call it; ends with a barrier.
__device__ __forceinline__ void eng_row_table(const EngineJob& J, int64_t b, int64_t e, int32_t* tab, int32_t total,
                                              bool groups) {
  for (int32_t i = threadIdx.x; i < total; i += blockDim.x) tab[i] = 0;
  __syncthreads();
  for (int64_t x = b + threadIdx.x; x < e; x += blockDim.x) atomicAdd(&tab[J.pi[J.g.adj[x]]], J.g.adjw[x]);
  __syncthreads();
  if (groups) conn_groups(J.topo, J.gl, tab);
}

struct PlainGather {  // neighbour PEs through plain loads (the mapping changes inside the launch)
  const int32_t* pi;
  __device__ __forceinline__ int32_t operator()(int32_t u) const { return pi[u]; }
};

// Stages one tile of neighbour PEs and returns T(P(v)) = sum_j w_j D(P(v), c_j)
// of the lane's vertex; `cand` tells whether a staged row has a neighbour
// outside P(v) (oversized tiles are left to the global path: cand false).
// A row of more than kEngLaneDeg entries gives 0 and no candidate here.
template <int kTE>
__device__ __forceinline__ TileLane eng_stage(const EngineJob& J, const TileGraph& tg, int64_t tile, int lane,
                                              int32_t* sc, int32_t* sw, const int32_t* sdist, int64_t& Tp,
                                              bool& cand, bool all_tp) {
  const TileLane t = stage_tile<kTE>(tg, tile * kTileV, lane, sc, sw, PlainGather{J.pi});
  Tp = 0;
  cand = false;
  if (t.v < tg.n && !eng_heavy(J, t.e - t.b)) {
    const int deg = (int)(t.e - t.b);
    const int32_t p = J.pi[t.v];
    if (t.staged) {
      const int32_t* c = sc + (t.b - t.E0);
      const int32_t* w = sw + (t.b - t.E0);
      for (int j = 0; j < deg; j++) cand |= c[j] != p;
      if (cand || all_tp)
        for (int j = 0; j < deg; j++) Tp += (int64_t)w[j] * dcode(sdist, p, c[j]);
    } else {
      Tp = row_cost(PlainRow{tg.adj + t.b, tg.adjw + t.b, J.pi}, deg, sdist, p);
    }
  }
  return t;
}

// Alg. 5 destinations of the lanes in `work` (vertices of an overloaded block
// that are not heavy) from their staged rows, four at a time by 8-lane
// sub-warps: the neighbouring block q != A with W(q) <= sigma of largest
// score, lowest id on ties.  The score is conn(v, q) for the cut gains, or
// -T(q) = -sum_u w D(q, P(u)) for the J gains (kJ).  out(lane, A, found, q,
// score of A, score of q, staged codes, staged weights, degree) runs on the
// sub-warp's first lane; the gain is the difference of the two scores.
template <bool kJ, class Out>
__device__ __forceinline__ void reb_tile_queue(unsigned work, const TileLane& tl, int32_t A, const int32_t* sc,
                                               const int32_t* sw, const int64_t* W, int64_t sigma,
                                               const int32_t* sdist, int lane, Out out) {
  const int sub = lane >> 3, sl = lane & 7;
  const int rounds = (__popc(work) + 3) / 4;
  for (int r = 0; r < rounds; r++) {
    const int src = tile_worker(work, r, sub);
    const int s2 = src < 0 ? 0 : src;
    const int64_t vb = __shfl_sync(0xffffffffu, tl.b, s2);
    const int dg = (int)(__shfl_sync(0xffffffffu, tl.e, s2) - vb);
    const int32_t a = __shfl_sync(0xffffffffu, A, s2);
    const int32_t* c = sc + (vb - tl.E0);
    const int32_t* w = sw + (vb - tl.E0);
    if constexpr (!kJ) {
      int32_t ca = 0, bconn = -1, bc = INT32_MAX;
      if (src >= 0) {
        for (int j = sl; j < dg; j += kSubWarp) {
          const int32_t q = c[j];
          if (q == a) {
            ca += w[j];
            continue;
          }
          if (W[q] > sigma) continue;
          bool seen = false;
          for (int l = 0; l < j; l++)
            if (c[l] == q) {
              seen = true;
              break;
            }
          if (seen) continue;
          int32_t cc = 0;
          for (int l = j; l < dg; l++) cc += (c[l] == q) ? w[l] : 0;
          if (cc > bconn || (cc == bconn && q < bc)) {
            bconn = cc;
            bc = q;
          }
        }
      }
#pragma unroll
      for (int o = kSubWarp / 2; o > 0; o >>= 1) {
        ca += __shfl_xor_sync(0xffffffffu, ca, o);
        const int32_t oc = __shfl_xor_sync(0xffffffffu, bconn, o);
        const int32_t oq = __shfl_xor_sync(0xffffffffu, bc, o);
        if (oc > bconn || (oc == bconn && oq < bc)) {
          bconn = oc;
          bc = oq;
        }
      }
      if (src >= 0 && sl == 0) out(src, a, bconn >= 0, bc, (int64_t)ca, (int64_t)bconn, c, w, dg);
    } else {
      int64_t ca = 0, bconn = 0;
      int32_t bc = INT32_MAX;
      bool found = false;
      if (src >= 0) {
        for (int j = sl; j < dg; j += kSubWarp) {
          const int32_t q = c[j];
          ca -= (int64_t)w[j] * dcode(sdist, a, q);
          if (q == a || W[q] > sigma) continue;
          bool seen = false;
          for (int l = 0; l < j; l++)
            if (c[l] == q) {
              seen = true;
              break;
            }
          if (seen) continue;
          int64_t cc = 0;
          for (int l = 0; l < dg; l++) cc -= (int64_t)w[l] * dcode(sdist, q, c[l]);
          if (!found || cc > bconn || (cc == bconn && q < bc)) {
            bconn = cc;
            bc = q;
            found = true;
          }
        }
      }
#pragma unroll
      for (int o = kSubWarp / 2; o > 0; o >>= 1) {
        ca += __shfl_xor_sync(0xffffffffu, ca, o);
        const int64_t oc = __shfl_xor_sync(0xffffffffu, bconn, o);
        const int32_t oq = __shfl_xor_sync(0xffffffffu, bc, o);
        const bool of = __shfl_xor_sync(0xffffffffu, found, o);
        if (of && (!found || oc > bconn || (oc == bconn && oq < bc))) {
          bconn = oc;
          bc = oq;
          found = true;
        }
      }
      if (src >= 0 && sl == 0) out(src, a, found, bc, ca, bconn, c, w, dg);
    }
  }
}

// Inclusive prefix sum over the 32 lanes of a warp.
__device__ __forceinline__ int64_t warp_incl_scan(int64_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exact change of J by the moves of an LP or weak step, added to the J
// accumulator (the mapping still holds the old values): the movers of each
// warp tile are served four at a time by 8-lane sub-warps, the movers with
// more than kEngLaneDeg entries by whole CTAs.
template <class Mv>
__device__ void eng_delta(const EngineJob& J, const Mv& mv, EngSmem& S, const EngGeom& eg, int64_t ntiles) {
  const GraphView& g = J.g;
  const int lane = eg.lane, sub = lane >> 3, sl = lane & 7;
  int64_t acc = 0;
  for (int64_t tile = eg.gw; tile < ntiles; tile += eg.GW) {
    const int64_t v = tile * kTileV + lane;
    const unsigned work =
        __ballot_sync(0xffffffffu, v < g.n && mv.moved(v) && !eng_heavy_row(J, v));
    const int rounds = (__popc(work) + 3) / 4;
    for (int r = 0; r < rounds; r++) {
      const int src = tile_worker(work, r, sub);
      if (src < 0) continue;
      const int64_t vv = tile * kTileV + src;
      const int32_t ov = J.pi[vv], nv = mv.target(vv);
      const int64_t xe = g.xadj[vv + 1];
      for (int64_t x = g.xadj[vv] + sl; x < xe; x += kSubWarp)
        acc += delta_entry(mv, J.pi, S.sdist, ov, nv, g.adj[x], g.adjw[x]);
    }
    __syncwarp();
  }
  eng_heavy_rows(J, eg, [&](int32_t v, int64_t b, int64_t e) {
    if (!mv.moved(v)) return;
    const int32_t ov = J.pi[v], nv = mv.target(v);
    for (int64_t x = b + threadIdx.x; x < e; x += blockDim.x)
      acc += delta_entry(mv, J.pi, S.sdist, ov, nv, g.adj[x], g.adjw[x]);
  });
  acc = block_sum(acc, S.sm);
  if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)J.Jacc, (unsigned long long)acc);
}

// Shared-memory layout of the rebalancing steps in the engine's dynamic
// shared memory: the cut bucket and remainder of every block (code spaces up
// to kEngCutSmem) and the short-list resolution behind them; the sorts of the
// first CTA reuse the area once the cuts are no longer read from it.
constexpr int kEngCutSmem = 4096;
static_assert(kEngCutSmem * 12 + kEngThreads * (8 + 8 + 4 + 8 + 1) <= 2 * kSmallSort * 12,
              "cut tables and short-list resolution fit in the engine's smallest dynamic shared memory");

// weak step, short list: movers are the selected vertices below the cut
// bucket and those of the cut bucket that the CTA's own resolution selected
struct WeakMovesShared {
  const uint8_t* elig;
  const uint8_t* sel;   // 1: below the cut bucket, 2: in the list (decision in s_sel)
  const int32_t* dest;
  const int64_t* slot;  // list slot of a vertex marked 2
  const uint8_t* s_sel;
  __device__ __forceinline__ bool moved(int64_t v) const {
    if (!elig[v]) return false;
    const uint8_t s = sel[v];
    return s == 1 || (s == 2 && s_sel[slot[v]]);
  }
  __device__ __forceinline__ int32_t target(int64_t v) const { return dest[v]; }
};

// Resolution of a cut-bucket list of at most blockDim entries by the calling
// CTA: rank sort by (block, id), exclusive prefix of the weights in that
// order, selection while the weight before a vertex in its block's bucket is
// below the block's remainder.  Returns the decisions by list slot (shared).
__device__ uint8_t* eng_resolve_local(const EngineJob& J, EngSmem& S, int32_t* area, int ln, int idbits,
                                      const int64_t* rem) {
  uint64_t* rk = reinterpret_cast<uint64_t*>(area);  // keys by slot
  uint64_t* ok = rk + kEngThreads;                   // keys in order
  int32_t* os = reinterpret_cast<int32_t*>(ok + kEngThreads);  // slots in order
  int64_t* ex = reinterpret_cast<int64_t*>(os + kEngThreads);  // exclusive prefix in order
  uint8_t* s_sel = reinterpret_cast<uint8_t*>(ex + kEngThreads);
  const int i = threadIdx.x;
  const uint64_t idmask = (1ULL << idbits) - 1ULL;
  uint64_t ki = 0;
  if (i < ln) {
    ki = J.key0[i];
    rk[i] = ki;
  }
  __syncthreads();
  if (i < ln) {
    int r = 0;  // keys are distinct (one per vertex)
    for (int j = 0; j < ln; j++) r += rk[j] < ki ? 1 : 0;
    ok[r] = ki;
    os[r] = i;
  }
  __syncthreads();
  const int64_t c = i < ln ? (int64_t)J.g.vw[(int64_t)(ok[i] & idmask)] : 0;
  int64_t tot;
  const int64_t e = block_exclusive_scan(c, S.sm, &tot);
  ex[i] = e;
  __syncthreads();
  if (i < ln) {
    const uint64_t A = ok[i] >> idbits;
    int h = i;
    while (h > 0 && (ok[h - 1] >> idbits) == A) h--;  // first entry of the block
    s_sel[os[i]] = (e - ex[h] < rem[A]) ? 1 : 0;
  }
  __syncthreads();
  return s_sel;
}

// Alg. 6 on one job by the calling cluster (all its threads call it).
// kVar: the job may use the refinement variants (relaxed filter, J gains in
// rebalancing); the plain instantiation leaves their code out.
template <int kTE, bool kVar, class Sync>
__device__ void engine_run_job(const EngineJob& J, EngSmem& S, int32_t* dyn, int32_t* sc, int32_t* sw,
                               const EngGeom& eg, const Sync& sy) {
  const GraphView g = J.g;
  const int32_t n = g.n;
  const int64_t gt = eg.gt, GT = eg.GT;
  const int lane = eg.lane;
  const bool lead = eg.lead;
  const TileGraph tg{n, g.xadj, g.adj, g.adjw};
  const int64_t ntiles = ((int64_t)n + kTileV - 1) / kTileV;
  // with at most one tile per warp, the entries staged for J stay valid for
  // the gain pass of the same iteration (the mapping does not change between)
  const bool single = ntiles <= eg.GW;
  RefineState* s = J.s;
  __syncthreads();
  load_sdist(S.sdist, J.topo);
  __syncthreads();

  // --- initial state: block weights, locks, best copy, J, controller ---
  if (lead)
    for (int32_t b = threadIdx.x; b < J.topo.kc; b += blockDim.x) J.W[b] = 0;
  if (lead && threadIdx.x == 0) {
    RefineState z{};
    z.rounds = J.rounds;
    z.level = J.level;
    *s = z;
    *J.Jacc = 0;
  }
  sy.sync();
  for (int64_t v = gt; v < n; v += GT) {
    atomicAdd((unsigned long long*)&J.W[J.pi[v]], (unsigned long long)(int64_t)g.vw[v]);
    J.lock[v] = 0;
    J.best[v] = J.pi[v];
  }
  int phase = 0;
  int32_t prev_kind = KIND_NONE;
  TileLane t0{};
  int64_t Tp0 = 0;
  bool cand0 = false;
  while (true) {
    // J of the current mapping (after an LP or weak step the accumulator
    // already holds it: old J plus the step's exact change), then the Alg. 6
    // decision
    const bool full = phase == 0 || !(prev_kind == KIND_LP || prev_kind == KIND_WEAK);
    const bool reuse = single && full;  // the gain pass may use this pass's staged tiles
    if (full) {  // (uniform: the previous step's kind is known to every thread)
      int64_t acc = 0;
      for (int64_t tile = eg.gw; tile < ntiles; tile += eg.GW) {
        int64_t Tp;
        bool cand;
        const TileLane t = eng_stage<kTE>(J, tg, tile, lane, sc, sw, S.sdist, Tp, cand, true);
        acc += Tp;
        if (single) {
          t0 = t;
          Tp0 = Tp;
          cand0 = cand;
        }
        __syncwarp();
      }
      eng_heavy_rows(J, eg, [&](int32_t v, int64_t b, int64_t e) {
        const int32_t p = J.pi[v];
        for (int64_t x = b + threadIdx.x; x < e; x += blockDim.x)
          acc += (int64_t)g.adjw[x] * dcode(S.sdist, p, J.pi[g.adj[x]]);
      });
      acc = block_sum(acc, S.sm);
      if (threadIdx.x == 0 && acc) atomicAdd((unsigned long long*)J.Jacc, (unsigned long long)acc);
      sy.sync();
    }
    if (lead) {
      const int64_t mx = block_max_w(J.W, J.topo.kc, S.smax);
      if (threadIdx.x == 0) {
        const int64_t Jv = *(volatile int64_t*)J.Jacc;
        control_step(s, mx, Jv, J.ctl, phase, 0, 0);
        *J.Jacc = next_j_base(s, Jv);
        J.cnt[CNT_ELIG] = 0;  // the cut-bucket list of a rebalancing step
      }
      __syncthreads();
      // a rebalancing step: its threshold sigma and destination list U now
      const int32_t next = *(volatile int32_t*)&s->kind;
      if (next == KIND_WEAK || next == KIND_STRONG) {
        const RebPrepArgs pa{J.W, J.pe_of_code, J.topo, J.lmax, J.cV, J.sigma_gap, J.U, J.cnt, J.accepted};
        reb_prep_body(pa, next == KIND_STRONG);
      }
    }
    sy.sync();
    const int32_t done = *(volatile int32_t*)&s->done;
    const int32_t kind = *(volatile int32_t*)&s->kind;
    const int32_t copy = *(volatile int32_t*)&s->copy_best;
    if (copy)
      for (int64_t v = gt; v < n; v += GT) J.best[v] = J.pi[v];
    if (done) break;
    phase = 1;
    prev_kind = kind;
    if (kind == KIND_LP) {
      // Alg. 4 step 1: staged tiles, lane check, sub-warp work queue
      for (int64_t tile = eg.gw; tile < ntiles; tile += eg.GW) {
        TileLane t = t0;
        int64_t Tp = Tp0;
        bool cand = cand0;
        if (!reuse) t = eng_stage<kTE>(J, tg, tile, lane, sc, sw, S.sdist, Tp, cand, false);
        int32_t p = -1;
        if (t.v < n && !eng_heavy(J, t.e - t.b)) {
          p = J.pi[t.v];
          bool written = false;
          if (J.lock[t.v]) {
            J.lock[t.v] = 0;
            cand = false;
          } else if (!t.staged) {  // oversized tile: this lane alone, from global memory
            const PlainRow r{g.adj + t.b, g.adjw + t.b, J.pi};
            int32_t bc;
            int64_t bt;
            if (best_target(r, (int)(t.e - t.b), p, S.sdist, bc, bt) &&
                (kVar ? J.flt.admit(Tp - bt, J.flt.num > 0 ? row_own(r, (int)(t.e - t.b), p) : 0)
                      : Tp - bt >= 0)) {
              J.inx[t.v] = 1;
              J.pp[t.v] = bc;
              J.gain[t.v] = Tp - bt;
              written = true;
            }
          }
          if (!cand && !written) {
            J.inx[t.v] = 0;
            J.pp[t.v] = p;
            J.gain[t.v] = 0;
          }
        }
        const unsigned work = __ballot_sync(0xffffffffu, cand);
        tile_gain_queue(work, t, p, Tp, sc, sw, kTE, NoRowLoader{}, S.sdist, lane, kVar && J.flt.num > 0,
                        [&](int src, int64_t Gv, int32_t bc, int32_t pv, int64_t own) {
          const int64_t v = tile * kTileV + src;
          const bool in = kVar ? J.flt.admit(Gv, own) : Gv >= 0;
          J.inx[v] = in ? 1 : 0;
          J.pp[v] = in ? bc : pv;
          J.gain[v] = in ? Gv : 0;
        });
        __syncwarp();
      }
      if (J.has_heavy) {
        __syncthreads();  // the warps' staging areas are free for the row tables
        const LpFilter flt = kVar ? J.flt : LpFilter{0, 1};
        eng_heavy_rows(J, eg, [&](int32_t v, int64_t b, int64_t e) {
          const int32_t p = J.pi[v];
          if (J.lock[v]) {
            __syncthreads();  // every thread has read the lock
            if (threadIdx.x == 0) {
              J.lock[v] = 0;
              J.inx[v] = 0;
              J.pp[v] = p;
              J.gain[v] = 0;
            }
            return;
          }
          eng_row_table(J, b, e, dyn, J.gl.total, true);
          lp_hub_decide(dyn, J.topo, J.gl, flt, v, p, J.pp, J.gain, J.inx, S.hb, S.hc);
        });
      }
      sy.sync();
      // step 2: recomputed gain under ord, one 8-lane sub-warp per candidate
      for (int64_t tile = eg.gw; tile < ntiles; tile += eg.GW) {
        const int64_t v = tile * kTileV + lane;
        const unsigned work =
            __ballot_sync(0xffffffffu, v < n && J.inx[v] && !eng_heavy_row(J, v));
        const int sub = lane >> 3, sl = lane & 7;
        const int rounds = (__popc(work) + 3) / 4;
        for (int r = 0; r < rounds; r++) {
          const int src = tile_worker(work, r, sub);
          const int64_t vv = tile * kTileV + (src < 0 ? 0 : src);
          int64_t sum = 0;
          if (src >= 0) {
            const int32_t p = J.pi[vv], q = J.pp[vv];
            const int64_t gv = J.gain[vv];
            const int64_t xe = g.xadj[vv + 1];
            for (int64_t x = g.xadj[vv] + sl; x < xe; x += kSubWarp) {
              const int32_t u = g.adj[x];
              int32_t bu = J.pi[u];
              if (J.inx[u]) {
                const int64_t gu = J.gain[u];
                if (gu > gv || (gu == gv && u < vv)) bu = J.pp[u];
              }
              sum += (int64_t)g.adjw[x] * (dcode(S.sdist, p, bu) - dcode(S.sdist, q, bu));
            }
          }
#pragma unroll
          for (int o = kSubWarp / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (src >= 0 && sl == 0 && sum >= 0) J.lock[vv] = 1;
        }
        __syncwarp();
      }
      eng_heavy_rows(J, eg, [&](int32_t v, int64_t b, int64_t e) {
        if (!J.inx[v]) return;
        const int32_t p = J.pi[v], q = J.pp[v];
        const int64_t gv = J.gain[v];
        int64_t sum = 0;
        for (int64_t x = b + threadIdx.x; x < e; x += blockDim.x) {
          const int32_t u = g.adj[x];
          int32_t bu = J.pi[u];
          if (J.inx[u]) {
            const int64_t gu = J.gain[u];
            if (gu > gv || (gu == gv && u < v)) bu = J.pp[u];
          }
          sum += (int64_t)g.adjw[x] * (dcode(S.sdist, p, bu) - dcode(S.sdist, q, bu));
        }
        sum = block_sum(sum, S.sm);
        if (threadIdx.x == 0 && sum >= 0) J.lock[v] = 1;
      });
      sy.sync();
      eng_delta(J, LpMoves{J.lock, J.pp}, S, eg, ntiles);
      sy.sync();
      // step 3: simultaneous move of M
      for (int64_t v = gt; v < n; v += GT) {
        if (!J.lock[v]) continue;
        const int32_t p = J.pi[v], q = J.pp[v];
        const int64_t c = g.vw[v];
        J.pi[v] = q;
        atomicAdd((unsigned long long*)&J.W[p], (unsigned long long)(-c));
        atomicAdd((unsigned long long*)&J.W[q], (unsigned long long)c);
      }
      sy.sync();
      continue;
    }
    // --- weak / strong rebalancing ---
    const bool strong = kind == KIND_STRONG;
    const int32_t t = *(volatile int32_t*)&s->t;
    const int64_t sigma = *(volatile int64_t*)&J.cnt[CNT_SIGMA];
    const int64_t nU = *(volatile int64_t*)&J.cnt[CNT_NU];
    // eligible vertices and their destinations: lane check, then staged rows
    for (int64_t tile = eg.gw; tile < ntiles; tile += eg.GW) {
      const int64_t v = tile * kTileV + lane;
      int32_t A = -1;
      bool cand = false;
      if (v < n && !eng_heavy_row(J, v)) {
        A = J.pi[v];
        const int64_t WA = J.W[A];
        cand = WA > J.lmax && 2 * (int64_t)J.k * g.vw[v] <= 3 * ((int64_t)J.k * WA - J.cV);
        if (!cand) J.elig[v] = 0;
      }
      if (__ballot_sync(0xffffffffu, cand) == 0) continue;
      const TileLane tl = stage_tile<kTE>(tg, tile * kTileV, lane, sc, sw, PlainGather{J.pi});
      if (cand && !tl.staged) {  // oversized tile: this lane alone, from global memory
        int32_t dst, bk;
        bool ok;
        if constexpr (kVar)
          ok = J.reb_obj != 0 ? eng_reb_select<true>(J, (int32_t)v, sigma, nU, t, S.sdist, dst, bk)
                              : eng_reb_select<false>(J, (int32_t)v, sigma, nU, t, S.sdist, dst, bk);
        else
          ok = eng_reb_select<false>(J, (int32_t)v, sigma, nU, t, S.sdist, dst, bk);
        J.elig[v] = ok ? 1 : 0;
        if (ok) {
          J.dest[v] = dst;
          J.bkt[v] = (uint8_t)bk;
          atomicAdd((unsigned long long*)&J.tab[(int64_t)A * kBuckets + bk], (unsigned long long)(int64_t)g.vw[v]);
        }
        cand = false;
      }
      const unsigned work = __ballot_sync(0xffffffffu, cand);
      auto reb_out = [&](int src, int32_t a, bool found, int32_t bc, int64_t sa, int64_t sb, const int32_t* rc,
                         const int32_t* rw, int dg) {
                       const int64_t u = tile * kTileV + src;
                       int64_t gcut;
                       int32_t dst;
                       if (found) {
                         gcut = sb - sa;
                         dst = bc;
                       } else if (nU > 0) {
                         dst = J.U[h_rebalance(J.seed, J.level, t, u) % (uint64_t)nU];
                         int64_t sr = 0;  // the drawn block is not a neighbour: conn 0, or -T(q)
                         if (kVar && J.reb_obj)
                           for (int l = 0; l < dg; l++) sr -= (int64_t)rw[l] * dcode(S.sdist, dst, rc[l]);
                         gcut = sr - sa;
                       } else {
                         J.elig[u] = 0;
                         return;
                       }
                       const int bk = loss_bucket(gcut);
                       J.elig[u] = 1;
                       J.dest[u] = dst;
                       J.bkt[u] = (uint8_t)bk;
                       atomicAdd((unsigned long long*)&J.tab[(int64_t)a * kBuckets + bk],
                                 (unsigned long long)(int64_t)g.vw[u]);
                     };
      if (kVar && J.reb_obj != 0)
        reb_tile_queue<true>(work, tl, A, sc, sw, J.W, sigma, S.sdist, lane, reb_out);
      else
        reb_tile_queue<false>(work, tl, A, sc, sw, J.W, sigma, S.sdist, lane, reb_out);
      __syncwarp();
    }
    if (J.has_heavy) {
      __syncthreads();  // the warps' staging areas are free for the row tables
      const RebArgs ra{J.W, J.U, J.cnt, J.tab, J.lmax, J.cV, J.k, J.seed, kVar ? J.reb_obj : 0, J.topo};
      eng_heavy_rows(J, eg, [&](int32_t v, int64_t b, int64_t e) {
        const int32_t A = J.pi[v];
        if (!reb_eligible(ra, A, g.vw[v])) {
          if (threadIdx.x == 0) J.elig[v] = 0;
          return;
        }
        eng_row_table(J, b, e, dyn, ra.obj ? J.gl.total : J.topo.kc, ra.obj != 0);
        reb_hub_decide(dyn, ra, J.topo.kc, J.gl, v, A, g.vw[v], J.dest, J.bkt, J.elig, s, S.hb, S.hc);
      });
    }
    sy.sync();
    // the cut bucket of each overloaded block A: the first bucket whose
    // inclusive prefix of eligible weight exceeds W(A) - L_max (one warp per
    // block, buckets lane and 32 + lane)
    static_assert(kBuckets == 64, "two buckets per lane");
    const int idbits = bits_for_n(n);
    const int32_t kc = J.topo.kc;
    auto warp_cut = [&](int64_t A, bool zero, int32_t* bcut_out, int64_t* rem_out) {
      const int64_t WA = J.W[A];
      if (WA <= J.lmax) return;
      const int64_t E = WA - J.lmax;
      int64_t* row = J.tab + A * kBuckets;
      const int64_t x0 = row[lane], x1 = row[32 + lane];
      if (zero) {
        row[lane] = 0;
        row[32 + lane] = 0;
      }
      const int64_t p0 = warp_incl_scan(x0, lane);
      const int64_t p1 = warp_incl_scan(x1, lane) + __shfl_sync(0xffffffffu, p0, 31);
      const unsigned m0 = __ballot_sync(0xffffffffu, p0 > E), m1 = __ballot_sync(0xffffffffu, p1 > E);
      const int cut = m0 ? __ffs(m0) - 1 : (m1 ? 32 + __ffs(m1) - 1 : kBuckets);
      const int pl = cut - 1;  // exclusive prefix of the cut bucket
      const int64_t q0 = __shfl_sync(0xffffffffu, p0, pl < 0 ? 0 : (pl & 31));
      const int64_t q1 = __shfl_sync(0xffffffffu, p1, pl < 32 ? 0 : (pl & 31));
      const int64_t excl = pl < 0 ? 0 : (pl < 32 ? q0 : q1);
      if (lane == 0) {
        bcut_out[A] = cut;
        rem_out[A] = cut < kBuckets ? E - excl : 0;
      }
    };
    // With a small code space every CTA computes the cuts itself into shared
    // memory (no barrier before the classification; the bucket totals are
    // cleared after the next barrier); else one warp per block, cluster-wide.
    const bool cut_local = kc <= kEngCutSmem;
    int64_t* s_rem = reinterpret_cast<int64_t*>(dyn);
    int32_t* s_bcut = reinterpret_cast<int32_t*>(s_rem + kEngCutSmem);
    if (cut_local) {
      for (int64_t A = threadIdx.x >> 5; A < kc; A += blockDim.x >> 5) warp_cut(A, false, s_bcut, s_rem);
      __syncthreads();
    } else {
      for (int64_t A = eg.gw; A < kc; A += eg.GW) warp_cut(A, true, J.bcut, J.rem);
      sy.sync();
    }
    const int32_t* bcut = cut_local ? s_bcut : J.bcut;
    const int64_t* rem = cut_local ? s_rem : J.rem;  // (the first CTA may switch to J.rem below)
    // below the cut bucket: moves; above: stays; in it: appended to the list
    // (in a weak step marked 2, with its list slot)
    for (int64_t v = gt; v < n; v += GT) {
      if (!J.elig[v]) continue;
      const int32_t A = J.pi[v];
      const int32_t bb = J.bkt[v], cut = bcut[A];
      if (bb != cut) {
        J.sel[v] = bb < cut ? 1 : 0;
        continue;
      }
      J.sel[v] = 0;
      if (rem[A] > 0) {
        const unsigned long long i = atomicAdd((unsigned long long*)&J.cnt[CNT_ELIG], 1ULL);
        J.key0[i] = ((uint64_t)(uint32_t)A << idbits) | (uint64_t)v;
        J.val0[i] = (int32_t)v;
        if (!strong) {
          J.sel[v] = 2;
          J.sarr[v] = (int64_t)i;
        }
      }
    }
    sy.sync();
    if (cut_local && lead)  // the bucket totals for the next step
      for (int64_t i = threadIdx.x; i < (int64_t)kc * kBuckets; i += blockDim.x) J.tab[i] = 0;
    const int ln = (int)*(volatile int64_t*)&J.cnt[CNT_ELIG];
    if (!strong && cut_local && ln <= (int)blockDim.x) {
      // every CTA orders the short cut-bucket list by (block, id) itself and
      // keeps the decisions in shared memory: no barrier before the exact
      // change of J
      uint8_t* s_sel = eng_resolve_local(J, S, s_bcut + kEngCutSmem, ln, idbits, rem);
      const WeakMovesShared mv{J.elig, J.sel, J.dest, J.sarr, s_sel};
      eng_delta(J, mv, S, eg, ntiles);
      sy.sync();
      for (int64_t v = gt; v < n; v += GT) {
        if (!mv.moved(v)) continue;
        const int32_t p = J.pi[v], q = J.dest[v];
        const int64_t c = g.vw[v];
        J.pi[v] = q;
        atomicAdd((unsigned long long*)&J.W[p], (unsigned long long)(-c));
        atomicAdd((unsigned long long*)&J.W[q], (unsigned long long)c);
      }
      sy.sync();
      continue;
    }
    if (lead) {  // the cut-bucket list by (block, id), per-block prefix
      if (ln > 0) {
        if (cut_local) {  // the sort below reuses the shared memory of the cuts
          for (int64_t A = threadIdx.x; A < kc; A += blockDim.x) J.rem[A] = s_rem[A];
          __syncthreads();
        }
        rem = J.rem;
        const uint64_t* K;
        const int32_t* V;
        eng_sort(J, S, dyn, ln, J.topo.code_bits + idbits, K, V);
        cta_scan(
            ln, [&](int64_t i) { return (int64_t)g.vw[V[i]]; },
            [&](int64_t i, int64_t e, int64_t) {
              J.P[i] = e;
              if (i == 0 || (K[i] >> idbits) != (K[i - 1] >> idbits)) J.headP[K[i] >> idbits] = e;
            },
            S.sm);
        __syncthreads();
        for (int i = threadIdx.x; i < ln; i += blockDim.x) {
          const int32_t A = (int32_t)(K[i] >> idbits);
          J.sel[V[i]] = (J.P[i] - J.headP[A] < rem[A]) ? 1 : 0;
        }
      }
    }
    sy.sync();
    if (!strong) {
      eng_delta(J, WeakMoves{J.elig, J.sel, J.dest}, S, eg, ntiles);
      sy.sync();
      for (int64_t v = gt; v < n; v += GT) {
        if (!J.elig[v] || !J.sel[v]) continue;
        const int32_t p = J.pi[v], q = J.dest[v];
        const int64_t c = g.vw[v];
        J.pi[v] = q;
        atomicAdd((unsigned long long*)&J.W[p], (unsigned long long)(-c));
        atomicAdd((unsigned long long*)&J.W[q], (unsigned long long)c);
      }
      sy.sync();
      continue;
    }
    if (lead) {  // strong: destinations in (bucket, id) order, acceptance, water-filling
      const int64_t ns = cta_scan(
          n, [&](int64_t v) { return (int64_t)((J.elig[v] && J.sel[v]) ? 1 : 0); },
          [&](int64_t v, int64_t e, int64_t x) {
            if (x) {
              J.key0[e] = ((uint64_t)(uint32_t)J.dest[v] << kBucketBits) | J.bkt[v];
              J.val0[e] = (int32_t)v;
            }
          },
          S.sm);
      __syncthreads();
      const uint64_t* K = J.key0;
      const int32_t* V = J.val0;
      if (ns) eng_sort(J, S, dyn, (int)ns, J.topo.code_bits + kBucketBits, K, V);
      cta_scan(
          ns, [&](int64_t i) { return (int64_t)g.vw[V[i]]; },
          [&](int64_t i, int64_t e, int64_t) {
            J.P[i] = e;
            if (i == 0 || (K[i] >> kBucketBits) != (K[i - 1] >> kBucketBits)) J.headP[K[i] >> kBucketBits] = e;
          },
          S.sm);
      __syncthreads();
      for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
        const int32_t d = (int32_t)(K[i] >> kBucketBits);
        const int32_t v = V[i];
        const int64_t inc = J.P[i] + g.vw[v] - J.headP[d];
        const bool ok = J.W[d] + inc <= J.lmax;
        J.acc[v] = ok ? 1 : 0;
        if (ok) atomicAdd((unsigned long long*)&J.accepted[d], (unsigned long long)(int64_t)g.vw[v]);
      }
      __syncthreads();
      cta_scan(
          n,
          [&](int64_t v) { return (J.elig[v] && J.sel[v] && !J.acc[v]) ? (int64_t)g.vw[v] : (int64_t)0; },
          [&](int64_t v, int64_t e, int64_t x) {
            if (x) J.sarr[v] = e;
          },
          S.sm);
      const int32_t kc = J.topo.kc;
      const int64_t tot = cta_scan(
          kc,
          [&](int64_t b) {
            int64_t r = 0;
            if (J.pe_of_code[b] >= 0 && J.W[b] <= J.lmax) {
              r = J.lmax - J.W[b] - J.accepted[b];
              if (r < 0) r = 0;
            }
            return r;
          },
          [&](int64_t b, int64_t e, int64_t) { J.Rb[b] = e; }, S.sm);
      if (threadIdx.x == 0) J.Rb[kc] = tot;
      __syncthreads();
      for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
        const int32_t v = V[i];
        const int64_t c = g.vw[v];
        int32_t q = -1;
        if (J.acc[v]) {
          q = (int32_t)(K[i] >> kBucketBits);
        } else {
          const int64_t sv = J.sarr[v];
          int32_t lo = 0, hi = kc + 1;
          while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (J.Rb[mid] <= sv) lo = mid + 1;
            else hi = mid;
          }
          const int32_t bb = lo - 1;
          if (bb >= 0 && bb < kc && sv + c <= J.Rb[bb + 1]) q = bb;
        }
        if (q < 0) continue;
        const int32_t p = J.pi[v];
        J.pi[v] = q;
        atomicAdd((unsigned long long*)&J.W[p], (unsigned long long)(-c));
        atomicAdd((unsigned long long*)&J.W[q], (unsigned long long)c);
      }
    }
    sy.sync();
  }
  for (int64_t v = gt; v < n; v += GT) J.pi[v] = J.best[v];
}

template <int kTE, bool kVar>
__global__ void __launch_bounds__(kEngThreads, 1) k_engine(const EngineJob* __restrict__ jobs, int32_t njobs,
                                                          unsigned int* queue) {
  __shared__ EngSmem S;
  __shared__ int32_t job_slot;
  extern __shared__ __align__(16) int32_t eng_dyn[];
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int warp = threadIdx.x >> 5;
  EngGeom eg;
  eg.lane = threadIdx.x & 31;
  eg.lead = crank == 0;
  eg.gt = (int64_t)crank * blockDim.x + threadIdx.x;
  eg.GT = (int64_t)csize * blockDim.x;
  eg.gw = (int64_t)crank * (blockDim.x >> 5) + warp;
  eg.GW = (int64_t)csize * (blockDim.x >> 5);
  eg.cta = crank;
  eg.ncta = csize;
  int32_t* sc = eng_dyn + warp * 2 * kTE;
  int32_t* sw = sc + kTE;
  if (!queue) {  // one job per cluster
    const int32_t jid = (int32_t)(blockIdx.x / csize);
    if (jid < njobs) engine_run_job<kTE, kVar>(jobs[jid], S, eng_dyn, sc, sw, eg, ClusterSync{});
    return;
  }
  // persistent clusters: the next job from the queue (jobs in the order given)
  while (true) {
    if (eg.lead && threadIdx.x == 0) job_slot = (int32_t)atomicAdd(queue, 1u);
    eng_sync();
    const int32_t jid = *cl.map_shared_rank(&job_slot, 0);
    eng_sync();
    if (jid >= njobs) break;
    engine_run_job<kTE, kVar>(jobs[jid], S, eng_dyn, sc, sw, eg, ClusterSync{});
  }
}

// The same engine over the whole grid (cooperative launch, one block per SM):
// for levels too large for one cluster, whose graph-launched iterations are
// dominated by launch gaps.
template <int kTE, bool kVar>
__global__ void __launch_bounds__(kEngThreads, 1) k_engine_grid(const EngineJob* __restrict__ job, GridBar* bar) {
  __shared__ EngSmem S;
  __shared__ unsigned int bar_flag;
  extern __shared__ __align__(16) int32_t eng_dyn[];
  const int warp = threadIdx.x >> 5;
  EngGeom eg;
  eg.lane = threadIdx.x & 31;
  eg.lead = blockIdx.x == 0;
  eg.gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  eg.GT = (int64_t)gridDim.x * blockDim.x;
  eg.gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  eg.GW = (int64_t)gridDim.x * (blockDim.x >> 5);
  eg.cta = (int)blockIdx.x;
  eg.ncta = (int)gridDim.x;
  int32_t* sc = eng_dyn + warp * 2 * kTE;
  int32_t* sw = sc + kTE;
  engine_run_job<kTE, kVar>(*job, S, eng_dyn, sc, sw, eg, GridSync{bar, &bar_flag, gridDim.x});
}

// Self-test of the bounded grid barrier: a barrier that waits for one more
// block than the grid has, so every wait runs out; the blocks then leave the
// kernel and the failure flag is set for the host.  Returns without output
// when the barrier was (wrongly) released.
__global__ void k_barrier_selftest(GridBar* bar, int* passed) {
  __shared__ unsigned int bar_flag;
  GridSync{bar, &bar_flag, gridDim.x + 1}.sync();
  if (threadIdx.x == 0) atomicAdd(passed, 1);  // not reached when the wait gives up
}

}  // namespace

// The strong variant continues from the selection made by launch_rebalance:
// selected movers in id order -> (destination, bucket, id) order -> accept
// while the destination stays within L_max -> water-fill the rejected ones.
static void launch_rebalance_strong_tail(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  const int64_t n = L.n;
  uint8_t* selflag = c.inx;
  int64_t* d_sel = c.counters + CNT_SEL;
  scan(LoadFlag2{c.elig, selflag}, StoreKeyed{c.dest, c.sel, c.sort.key[0], c.sort.val[0]}, n, nullptr, c.scan, c.st);
  k_copy_count<<<1, 1, 0, c.st>>>(c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(n)), d_sel); count_launch();
  k_strong_gate<<<1, 1, 0, c.st>>>(c.state, d_sel); count_launch();
  const int bits = c.topo.code_bits + kBucketBits;
  int cur = radix_sort_pairs(c.sort, n, d_sel, bits, c.st, &c.cap, &c.state->kernels);
  scan(LoadSortedWeight{c.sort.val[cur], L.vw}, StoreExcl{c.P64}, n, d_sel, c.scan, c.st);
  const unsigned g = grid_for(c, kThreads, n);
  k_heads<<<g, kThreads, 0, c.st>>>(c.sort.key[cur], c.P64, d_sel, n, c.headP); count_launch();
  k_reb_accept<<<g, kThreads, 0, c.st>>>(c.sort.key[cur], c.sort.val[cur], c.P64, c.headP, d_sel, n, c.W, c.lmax, L.vw,
                                         c.acc, c.accepted); count_launch();
  // rejected movers (selected, not accepted) in id order: prefix weights
  // (only for vertices in the selected list; acc is meaningful there)
  scan(LoadRejected{c.elig, selflag, c.acc, L.vw}, StoreIfPositive{c.sarr}, n, nullptr, c.scan, c.st);
  k_reb_residual<<<1, 1024, 0, c.st>>>(c.W, c.accepted, c.d_pe_of_code, c.topo.kc, c.lmax, c.Rb); count_launch();
  k_reb_apply_strong<<<g, kThreads, 0, c.st>>>(c.sort.key[cur], c.sort.val[cur], d_sel, n, c.acc, c.sarr, c.Rb,
                                               c.topo.kc, L.pi, L.vw, c.W, c.state); count_launch();
}

namespace {
CtlArgs ctl_args(Ctx& c) {
  return CtlArgs{c.lmax, c.topo.kc, c.cfg.patience, c.cfg.weak_max, c.cfg.phi_num, c.cfg.phi_den,
                 c.trace_kind, c.trace_J, c.trace_maxw, c.trace_cap};
}
}  // namespace

// Raises a kernel's dynamic shared memory limit to at least `bytes`.  The
// attribute belongs to the process, so contexts of different sizes must
// never lower it under one another: it only grows.
static void raise_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes at{};
  GM_CUDA(cudaFuncGetAttributes(&at, fn));
  if ((size_t)at.maxDynamicSharedSizeBytes < bytes)
    GM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

void refine_alloc(Ctx& c) {
  const size_t n = (size_t)std::max(1, c.n0);
  const size_t kc = (size_t)c.topo.kc;
  c.pp = c.mem.make<int32_t>(n);
  c.gain = c.mem.make<int64_t>(n);
  c.inx = c.mem.make<uint8_t>(n);
  c.lock = c.mem.make<uint8_t>(n);
  c.pi_best = c.mem.make<int32_t>(n);
  c.dest = c.mem.make<int32_t>(n);
  c.elig = c.mem.make<uint8_t>(n);
  c.sel = c.mem.make<uint8_t>(n);
  c.acc = c.mem.make<uint8_t>(n);
  c.sarr = c.mem.make<int64_t>(n);
  c.W = c.mem.make<int64_t>(kc);
  c.accepted = c.mem.make<int64_t>(kc);
  c.headP = c.mem.make<int64_t>(std::max(kc, n));
  c.Rb = c.mem.make<int64_t>(kc + 1);
  c.U = c.mem.make<int32_t>(kc);
  c.tab = c.mem.make<int64_t>(kc * kBuckets);
  c.bcut = c.mem.make<int32_t>(kc);
  c.rem = c.mem.make<int64_t>(kc);
  GM_CUDA(cudaMemsetAsync(c.tab, 0, kc * kBuckets * sizeof(int64_t), c.st));
  c.counters = c.mem.make<int64_t>(CNT_N);
  c.Jacc = c.mem.make<int64_t>(1);
  c.evctr = reinterpret_cast<unsigned int*>(c.mem.make<int64_t>(1));
  GM_CUDA(cudaMemsetAsync(c.evctr, 0, sizeof(int64_t), c.st));
  c.state = c.mem.make<RefineState>(1);
  c.probe_state = c.mem.make<RefineState>(1);
  GM_CUDA(cudaMemsetAsync(c.probe_state, 0, sizeof(RefineState), c.st));  // kind 0 = KIND_LP
  c.trace_kind = c.mem.make<int32_t>(c.trace_cap);
  c.trace_J = c.mem.make<int64_t>(c.trace_cap);
  c.trace_maxw = c.mem.make<int64_t>(c.trace_cap);
  GM_CUDA(cudaMemsetAsync(c.Jacc, 0, sizeof(int64_t), c.st));
  GM_CUDA(cudaMemsetAsync(c.lock, 0, n, c.st));
  GM_CUDA(cudaMemsetAsync(c.counters, 0, CNT_N * sizeof(int64_t), c.st));
  GM_CUDA(cudaMemsetAsync(c.state, 0, sizeof(RefineState), c.st));
  static_assert(sizeof(RefineState) <= kPinnedBlock, "pinned block too small");
  if (!c.h_state) c.h_state = static_cast<RefineState*>(pinned_get(sizeof(RefineState)));
  if (!c.h_small) c.h_small = static_cast<int64_t*>(pinned_get(8 * sizeof(int64_t)));
  c.gbar = c.mem.make<GridBar>(1);
  GM_CUDA(cudaMemsetAsync(c.gbar, 0, sizeof(GridBar), c.st));
  c.d_stats = c.mem.make<int64_t>(4);
  const size_t smem = conn_smem(c);
  if (smem > 48 * 1024) raise_smem((const void*)k_lp_gain_high, smem);
  static std::atomic<unsigned long long> resolve_done{0};  // one bit per device
  if (!(resolve_done.load() & (1ULL << (c.dev & 63)))) {
    GM_CUDA(cudaFuncSetAttribute(k_reb_resolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_sort_smem()));
    resolve_done.fetch_or(1ULL << (c.dev & 63));
  }
  const size_t reb_smem = (size_t)(c.cfg.reb_objective ? group_layout(c.topo).total : kc) * sizeof(int32_t);
  if (reb_smem > 48 * 1024) raise_smem((const void*)k_reb_select_high, reb_smem);
  if (kc * sizeof(int32_t) > 48 * 1024) raise_smem((const void*)k_block_weights, kc * sizeof(int32_t));
}

void compute_block_weights(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  GM_CUDA(cudaMemsetAsync(c.W, 0, (size_t)c.topo.kc * sizeof(int64_t), c.st));
  k_block_weights<<<grid_for(c, kThreads * 16, L.n), kThreads, (size_t)c.topo.kc * sizeof(int32_t), c.st>>>(
      L.n, L.pi, L.vw, c.topo.kc, c.W); count_launch();
  GM_CUDA(cudaGetLastError());
}

void objective(Ctx& c, int lvl, int64_t* J, int64_t* maxw) {
  compute_block_weights(c, lvl);
  GM_CUDA(cudaMemsetAsync(c.Jacc, 0, sizeof(int64_t), c.st));
  launch_eval(c, lvl);
  GM_CUDA(cudaGetLastError());
  std::vector<int64_t> W(c.topo.kc);
  int64_t hJ = 0;
  GM_CUDA(cudaMemcpyAsync(&hJ, c.Jacc, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(W.data(), c.W, W.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  if (J) *J = hJ;
  if (maxw) *maxw = W.empty() ? 0 : *std::max_element(W.begin(), W.end());
}

static void set_state(Ctx& c, int32_t kind, int32_t t, int32_t level) {
  RefineState s{};
  s.kind = kind;
  s.t = t;
  s.level = level;
  s.rounds = -1;
  *c.h_state = s;
  GM_CUDA(cudaMemcpyAsync(c.state, c.h_state, sizeof(RefineState), cudaMemcpyHostToDevice, c.st));
}

static int32_t read_moved(Ctx& c) {
  GM_CUDA(cudaMemcpyAsync(c.h_state, c.state, sizeof(RefineState), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  return c.h_state->moved;
}

int32_t lp_step(Ctx& c, int lvl) {
  compute_block_weights(c, lvl);
  set_state(c, KIND_LP, 0, lvl);
  launch_lp(c, lvl);
  GM_CUDA(cudaGetLastError());
  return read_moved(c);
}

int32_t rebalance_step(Ctx& c, int lvl, bool strong, int32_t t) {
  compute_block_weights(c, lvl);
  set_state(c, strong ? KIND_STRONG : KIND_WEAK, t, lvl);
  launch_rebalance(c, lvl);
  launch_rebalance_strong_tail(c, lvl);
  GM_CUDA(cudaGetLastError());
  return read_moved(c);
}

static void refine_stream(Ctx& c, int lvl, int32_t rounds, int64_t* J, int64_t* maxw, int32_t* iters) {
  Level& L = c.lv[lvl];
  compute_block_weights(c, lvl);
  GM_CUDA(cudaMemsetAsync(c.lock, 0, (size_t)std::max(1, L.n), c.st));
  GM_CUDA(cudaMemcpyAsync(c.pi_best, L.pi, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.st));
  RefineState s{};
  s.rounds = rounds;
  s.level = lvl;
  *c.h_state = s;
  GM_CUDA(cudaMemcpyAsync(c.state, c.h_state, sizeof(RefineState), cudaMemcpyHostToDevice, c.st));
  GM_CUDA(cudaMemsetAsync(c.Jacc, 0, sizeof(int64_t), c.st));
  const EvalCtl ec0{c.state, c.evctr, c.W, ctl_args(c), 0, 0, 0};
  const EvalCtl ec1{c.state, c.evctr, c.W, ctl_args(c), 1, 0, 0};
  launch_eval(c, lvl, &ec0);
  const unsigned gcopy = grid_for(c, kThreads * 4, L.n);
  while (true) {
    GM_CUDA(cudaMemcpyAsync(c.h_state, c.state, sizeof(RefineState), cudaMemcpyDeviceToHost, c.st));
    GM_CUDA(cudaStreamSynchronize(c.st));
    const RefineState h = *c.h_state;
    if (h.done) break;
    if (h.kind == KIND_LP) {
      launch_lp(c, lvl);
    } else {
      launch_rebalance(c, lvl);
      if (h.kind == KIND_STRONG) launch_rebalance_strong_tail(c, lvl);
    }
    launch_eval(c, lvl, &ec1, h.kind == KIND_STRONG);
    k_copy_best<<<gcopy, kThreads, 0, c.st>>>(c.state, L.pi, c.pi_best, L.n, IterCounts{0, 0, 0, 0}); count_launch();
    GM_CUDA(cudaGetLastError());
  }
  GM_CUDA(cudaMemcpyAsync(L.pi, c.pi_best, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.st));
  const RefineState h = *c.h_state;
  if (h.capped) throw ApiError(MAP_E_TIMEOUT, "refinement stopped at the iteration cap");
  c.last_iters = h.t;
  if (J) *J = h.best_J;
  if (maxw) *maxw = h.best_maxw;
  if (iters) *iters = h.t;
}

void drop_graph(Level& L) {
  if (L.gexec) cudaGraphExecDestroy(L.gexec);
  L.gexec = nullptr;
  L.g_rounds = -2;
  L.g_nhi = -1;
  L.g_nhuge = -1;
}

// Captures one level's whole Alg. 6 run as a graph: initial J / weights, then
// WHILE(not done) { decide; IF(LP){Alg. 4}; IF(weak or strong){Alg. 5};
// IF(strong){strong tail}; J; control; copy best }, then best -> P.
static void build_refine_graph(Ctx& c, int lvl, int32_t rounds) {
  Level& L = c.lv[lvl];
  drop_graph(L);
  cudaStream_t saved = c.st;
  cap_streams(c);
  cudaStream_t cs = c.cap.s[0];
  const CtlArgs ca = ctl_args(c);
  const unsigned gcopy = grid_for(c, kThreads * 4, L.n);
  long long root = 0, n_fixed = 0, n_lp = 0, n_reb = 0, n_strong = 0;
  long long* outer = set_capture_counter(&root);
  GM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  c.cap.depth = 0;
  c.st = cs;
  try {
    GM_CUDA(cudaMemsetAsync(c.W, 0, (size_t)c.topo.kc * sizeof(int64_t), cs));
    k_block_weights<<<grid_for(c, kThreads * 16, L.n), kThreads, (size_t)c.topo.kc * sizeof(int32_t), cs>>>(
        L.n, L.pi, L.vw, c.topo.kc, c.W); count_launch();
    GM_CUDA(cudaMemsetAsync(c.lock, 0, (size_t)std::max(1, L.n), cs));
    GM_CUDA(cudaMemcpyAsync(c.pi_best, L.pi, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, cs));
    k_state_init<<<1, 1, 0, cs>>>(c.state, rounds, lvl); count_launch();
    GM_CUDA(cudaMemsetAsync(c.Jacc, 0, sizeof(int64_t), cs));
    cudaGraphConditionalHandle h_loop = cap_handle(cs, 0);
    const EvalCtl ec0{c.state, c.evctr, c.W, ca, 0, h_loop, 1};
    const EvalCtl ec1{c.state, c.evctr, c.W, ca, 1, h_loop, 1};
    launch_eval(c, lvl, &ec0);
    cap_cond(c.cap, cs, h_loop, cudaGraphCondTypeWhile, [&](cudaStream_t bs) {
      c.st = bs;
      set_capture_counter(&n_fixed);
      cudaGraphConditionalHandle h_lp = cap_handle(bs, 0), h_reb = cap_handle(bs, 0), h_strong = cap_handle(bs, 0);
      // counts of the bodies are known only after they are captured: the
      // decide node reads them from this iteration's parameters below
      k_decide_prep<<<1, 1024, 0, bs>>>(c.state, h_lp, h_reb, h_strong, reb_prep_args(c)); count_launch();
      set_capture_counter(&n_lp);
      cap_cond(c.cap, bs, h_lp, cudaGraphCondTypeIf, [&](cudaStream_t s2) {
        c.st = s2;
        launch_lp(c, lvl);
      });
      set_capture_counter(&n_reb);
      cap_cond(c.cap, bs, h_reb, cudaGraphCondTypeIf, [&](cudaStream_t s2) {
        c.st = s2;
        launch_rebalance(c, lvl, /*prep_done=*/true);
      });
      set_capture_counter(&n_strong);
      cap_cond(c.cap, bs, h_strong, cudaGraphCondTypeIf, [&](cudaStream_t s2) {
        c.st = s2;
        launch_rebalance_strong_tail(c, lvl);
      });
      set_capture_counter(&n_fixed);
      c.st = bs;
      launch_eval(c, lvl, &ec1);
      // this node is the iteration's last: all body counts are known now
      const IterCounts ic{(unsigned long long)n_fixed + 1, (unsigned long long)n_lp, (unsigned long long)n_reb,
                          (unsigned long long)n_strong};
      k_copy_best<<<gcopy, kThreads, 0, bs>>>(c.state, L.pi, c.pi_best, L.n, ic); count_launch();
      set_capture_counter(&root);
    });
    c.st = cs;
    GM_CUDA(cudaMemcpyAsync(L.pi, c.pi_best, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, cs));
    cudaGraph_t g = nullptr;
    GM_CUDA(cudaStreamEndCapture(cs, &g));
    c.cap.depth = -1;
    c.st = saved;
    set_capture_counter(outer);
    cudaError_t e = cudaGraphInstantiate(&L.gexec, g, 0);
    cudaGraphDestroy(g);
    GM_CUDA(e);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    c.cap.depth = -1;
    c.st = saved;
    set_capture_counter(outer);
    throw;
  }
  L.g_rounds = rounds;
  L.g_nhi = L.n_hi;
  L.g_nhuge = L.n_huge;
  L.g_root = root;
}

static void refine_graph(Ctx& c, int lvl, int32_t rounds, int64_t* J, int64_t* maxw, int32_t* iters) {
  Level& L = c.lv[lvl];
  if (!L.gexec || L.g_rounds != rounds || L.g_nhi != L.n_hi || L.g_nhuge != L.n_huge)
    build_refine_graph(c, lvl, rounds);
  GM_CUDA(cudaGraphLaunch(L.gexec, c.st));
  GM_CUDA(cudaMemcpyAsync(c.h_state, c.state, sizeof(RefineState), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  const RefineState h = *c.h_state;
  add_launches(L.g_root + (long long)h.kernels);
  if (h.capped) throw ApiError(MAP_E_TIMEOUT, "refinement stopped at the iteration cap");
  c.last_iters = h.t;
  if (J) *J = h.best_J;
  if (maxw) *maxw = h.best_maxw;
  if (iters) *iters = h.t;
}

// dynamic shared memory: the warps' staging arrays, or the two key / value
// buffers of the single-CTA sort (used at other times)
static size_t engine_smem(int te) {
  return std::max((size_t)(kEngThreads / 32) * 2 * te * sizeof(int32_t),
                  (size_t)2 * kSmallSort * (sizeof(uint64_t) + sizeof(int32_t)));
}

// Whether the engine takes every row of a level: the rows of more than
// kEngLaneDeg entries need their connectivity table (conn per PE code and the
// level group sums) in the dynamic shared memory of the smallest build.
static bool engine_rows_fit(const Ctx& c, const Level& L) {
  return L.max_deg <= kEngLaneDeg || (size_t)group_layout(c.topo).total * sizeof(int32_t) <= engine_smem(256);
}

// Cluster size of the fused engine for a level (0: not used).
static int engine_cluster(Ctx& c, const Level& L) {
  const int64_t lim = c.cfg.engine_max_n > 0 ? c.cfg.engine_max_n : (c.cfg.engine_max_n < 0 ? -1 : kEngMaxN);
  if (!c.use_graphs || c.prof || L.n > lim || !engine_rows_fit(c, L)) return 0;
  int C = (L.n + 1023) / 1024;  // about one vertex per thread
  if (C < 1) C = 1;
  if (C > c.eng_max_cluster) C = c.eng_max_cluster;
  return C;
}

using EngineKernel = void (*)(const EngineJob*, int32_t, unsigned int*);
// the variants exist for 512-entry tiles only
static EngineKernel engine_kernel(int te, bool var = false) {
  if (var) return k_engine<512, true>;
  return te == 256 ? k_engine<256, false> : k_engine<512, false>;
}
using GridKernel = void (*)(const EngineJob*, GridBar*);
static GridKernel grid_kernel(bool var) { return var ? k_engine_grid<512, true> : k_engine_grid<512, false>; }

static cudaLaunchConfig_t engine_config(int C, int te, unsigned grid, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kEngThreads);
  cfg.dynamicSmemBytes = engine_smem(te);
  cfg.stream = st;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = (unsigned)C;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Kernel attributes of both engine variants (once per process and device).
static void engine_attributes() {
  static std::mutex mu;
  static bool done[256] = {false};
  int dev = 0;
  GM_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 256 || done[dev]) return;
  for (bool var : {false, true})
    GM_CUDA(cudaFuncSetAttribute(grid_kernel(var), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)engine_smem(512)));
  for (int v = 0; v < 3; v++) {
    const int te = v == 0 ? 256 : 512;
    const EngineKernel k = engine_kernel(te, v == 2);
    GM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)engine_smem(te)));
    if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
  }
  done[dev] = true;
}

int engine_max_clusters(int C, int te) {
  engine_attributes();
  cudaLaunchAttribute attr{};
  cudaLaunchConfig_t cfg = engine_config(C, te, (unsigned)C, nullptr, &attr);
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)engine_kernel(te), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nclusters;
}

static void engine_setup(Ctx& c) {
  if (c.eng_max_cluster > 0) return;
  // the occupancy query is a property of the device: once per process
  static std::atomic<int> cached[64];
  const int d = c.dev & 63;
  int v = cached[d].load();
  if (v == 0) {
    v = engine_max_clusters(kEngMaxCluster, 512) > 0 ? kEngMaxCluster : 8;
    cached[d].store(v);
  }
  c.eng_max_cluster = v;
  if (!c.eng_job) {
    c.eng_job = c.mem.make<EngineJob>(1);
    static_assert(sizeof(EngineJob) <= kPinnedBlock, "pinned block too small");
    c.h_eng_job = pinned_get(sizeof(EngineJob));
  }
}

static EngineJob engine_job(Ctx& c, int lvl, int32_t rounds) {
  Level& L = c.lv[lvl];
  EngineJob j{};
  j.g = view(L);
  j.pi = L.pi;
  j.pp = c.pp;
  j.gain = c.gain;
  j.inx = c.inx;
  j.lock = c.lock;
  j.best = c.pi_best;
  j.dest = c.dest;
  j.elig = c.elig;
  j.bkt = c.sel;
  j.sel = c.inx;
  j.acc = c.acc;
  j.sarr = c.sarr;
  j.P = c.P64;
  j.W = c.W;
  j.accepted = c.accepted;
  j.U = c.U;
  j.tab = c.tab;
  j.bcut = c.bcut;
  j.rem = c.rem;
  j.headP = c.headP;
  j.Rb = c.Rb;
  j.key0 = c.sort.key[0];
  j.val0 = c.sort.val[0];
  j.key1 = c.sort.key[1];
  j.val1 = c.sort.val[1];
  j.cnt = c.counters;
  j.Jacc = c.Jacc;
  j.s = c.state;
  j.pe_of_code = c.d_pe_of_code;
  j.topo = c.topo;
  j.ctl = ctl_args(c);
  j.lmax = c.lmax;
  j.cV = c.cV;
  j.seed = c.cfg.seed;
  j.k = c.k;
  j.sigma_gap = c.cfg.sigma_gap;
  j.flt = LpFilter{c.cfg.lp_relax_num, c.cfg.lp_relax_den};
  j.reb_obj = c.cfg.reb_objective;
  j.level = lvl;
  j.rounds = rounds;
  j.hi = L.hi;
  j.n_hi = L.n_hi;
  j.has_heavy = L.max_deg > kEngLaneDeg ? 1 : 0;
  j.gl = group_layout(c.topo);
  return j;
}

size_t engine_job_bytes() { return sizeof(EngineJob); }

bool engine_job_write(Ctx& c, int lvl, int32_t rounds, void* dst) {
  engine_setup(c);
  const Level& L = c.lv[lvl];
  if (!engine_rows_fit(c, L)) return false;
  *static_cast<EngineJob*>(dst) = engine_job(c, lvl, rounds);
  return true;
}

void engine_launch(cudaStream_t st, const void* d_jobs, int njobs, unsigned int* queue, int C, int te,
                   int nclusters, bool var) {
  engine_attributes();
  if (var && te != 512) throw ApiError(MAP_E_INTERNAL, "the engine's variant build uses 512-entry tiles");
  cudaLaunchAttribute attr{};
  cudaLaunchConfig_t cfg = engine_config(C, te, (unsigned)(C * nclusters), st, &attr);
  GM_CUDA(cudaLaunchKernelEx(&cfg, engine_kernel(te, var), static_cast<const EngineJob*>(d_jobs), (int32_t)njobs,
                             queue));
  count_launch();
}

static void refine_engine(Ctx& c, int lvl, int32_t rounds, int C, int64_t* J, int64_t* maxw, int32_t* iters) {
  *static_cast<EngineJob*>(c.h_eng_job) = engine_job(c, lvl, rounds);
  GM_CUDA(cudaMemcpyAsync(c.eng_job, c.h_eng_job, sizeof(EngineJob), cudaMemcpyHostToDevice, c.st));
  engine_launch(c.st, c.eng_job, 1, nullptr, C, 512, 1, uses_variants(c.cfg));
  GM_CUDA(cudaMemcpyAsync(c.h_state, c.state, sizeof(RefineState), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  const RefineState h = *c.h_state;
  if (h.capped) throw ApiError(MAP_E_TIMEOUT, "refinement stopped at the iteration cap");
  c.last_iters = h.t;
  if (J) *J = h.best_J;
  if (maxw) *maxw = h.best_maxw;
  if (iters) *iters = h.t;
}

// Whether a level runs the grid-wide engine (levels above the cluster
// engine's size, up to grid_engine_max_n vertices).
static bool engine_grid_ok(Ctx& c, const Level& L) {
  const int64_t lim =
      c.cfg.grid_engine_max_n > 0 ? c.cfg.grid_engine_max_n : (c.cfg.grid_engine_max_n < 0 ? -1 : (1 << 18));
  if (!c.use_graphs || c.prof || L.n > lim || !engine_rows_fit(c, L)) return false;
  static std::atomic<int> cached[64];  // a property of the device: once per process
  if (c.eng_grid_blocks == 0) c.eng_grid_blocks = cached[c.dev & 63].load();
  if (c.eng_grid_blocks == 0) {
    int per_sm = 0;
    for (bool var : {false, true}) {  // both builds must fit the cooperative grid
      int ps = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, grid_kernel(var), kEngThreads, engine_smem(512)) !=
          cudaSuccess) {
        cudaGetLastError();
        ps = 0;
      }
      per_sm = var ? std::min(per_sm, ps) : ps;
    }
    if (per_sm < 1) per_sm = 0;
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c.dev);
    c.eng_grid_blocks = (coop && per_sm > 0) ? c.num_sms * per_sm : -1;
    cached[c.dev & 63].store(c.eng_grid_blocks);
  }
  return c.eng_grid_blocks > 0;
}

static void refine_engine_grid(Ctx& c, int lvl, int32_t rounds, int64_t* J, int64_t* maxw, int32_t* iters) {
  *static_cast<EngineJob*>(c.h_eng_job) = engine_job(c, lvl, rounds);
  GM_CUDA(cudaMemcpyAsync(c.eng_job, c.h_eng_job, sizeof(EngineJob), cudaMemcpyHostToDevice, c.st));
  GM_CUDA(cudaMemsetAsync(c.gbar, 0, sizeof(GridBar), c.st));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)c.eng_grid_blocks);
  cfg.blockDim = dim3(kEngThreads);
  cfg.dynamicSmemBytes = engine_smem(512);
  cfg.stream = c.st;
  cudaLaunchAttribute attr{};
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  GM_CUDA(cudaLaunchKernelEx(&cfg, grid_kernel(uses_variants(c.cfg)), static_cast<const EngineJob*>(c.eng_job),
                             static_cast<GridBar*>(c.gbar)));
  count_launch();
  GM_CUDA(cudaMemcpyAsync(c.h_state, c.state, sizeof(RefineState), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(c.h_small, c.gbar, sizeof(GridBar), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  if (reinterpret_cast<const GridBar*>(c.h_small)->err)
    throw ApiError(MAP_E_TIMEOUT, "a grid barrier of the refinement engine gave up waiting");
  const RefineState h = *c.h_state;
  if (h.capped) throw ApiError(MAP_E_TIMEOUT, "refinement stopped at the iteration cap");
  c.last_iters = h.t;
  if (J) *J = h.best_J;
  if (maxw) *maxw = h.best_maxw;
  if (iters) *iters = h.t;
}

// Runs the grid barrier self-test on stream st with a few blocks; returns
// whether the wait gave up (err set and no block passed the barrier).
bool barrier_selftest(cudaStream_t st) {
  GridBar* bar = nullptr;
  int* passed = nullptr;
  GM_CUDA(cudaMallocAsync(&bar, sizeof(GridBar), st));
  GM_CUDA(cudaMallocAsync(&passed, sizeof(int), st));
  GM_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBar), st));
  GM_CUDA(cudaMemsetAsync(passed, 0, sizeof(int), st));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(4);
  cfg.blockDim = dim3(128);
  cfg.stream = st;
  cudaLaunchAttribute attr{};
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  GM_CUDA(cudaLaunchKernelEx(&cfg, k_barrier_selftest, bar, passed));
  count_launch();
  GridBar hb{};
  int hp = -1;
  GM_CUDA(cudaMemcpyAsync(&hb, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaMemcpyAsync(&hp, passed, sizeof(int), cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  GM_CUDA(cudaFreeAsync(bar, st));
  GM_CUDA(cudaFreeAsync(passed, st));
  GM_CUDA(cudaStreamSynchronize(st));
  return hb.err != 0 && hp == 0;
}

void refine(Ctx& c, int lvl, int32_t rounds, int64_t* J, int64_t* maxw, int32_t* iters) {
  engine_setup(c);
  const int C = engine_cluster(c, c.lv[lvl]);
  if (C > 0 && c.sink) {
    RefineState h{};
    c.sink->refine(c, lvl, rounds, C, &h);
    if (h.capped) throw ApiError(MAP_E_TIMEOUT, "refinement stopped at the iteration cap");
    c.last_iters = h.t;
    if (J) *J = h.best_J;
    if (maxw) *maxw = h.best_maxw;
    if (iters) *iters = h.t;
  } else if (C > 0) refine_engine(c, lvl, rounds, C, J, maxw, iters);
  else if (engine_grid_ok(c, c.lv[lvl])) refine_engine_grid(c, lvl, rounds, J, maxw, iters);
  else if (c.use_graphs && !c.prof) refine_graph(c, lvl, rounds, J, maxw, iters);
  else refine_stream(c, lvl, rounds, J, maxw, iters);
}

// high-degree vertex list of a level (ascending ids)
namespace {
// Degree classes counted by one scan: the low 32 bits count the vertices of
// degree > kLowDeg, the high 32 bits those of degree > kMidDeg (a subset).
struct LoadHigh {
  const int64_t* xadj;
  int32_t mid_deg;
  __device__ int64_t operator()(int64_t v) const {
    const int64_t d = xadj[v + 1] - xadj[v];
    return (d > kLowDeg ? 1 : 0) + (d > mid_deg ? (1LL << 32) : 0);
  }
};
// hi[] gets every vertex of degree > kLowDeg; huge[] the positions in hi[] of
// those of degree > mid_deg
struct StoreHigh {
  int32_t* out;
  int32_t* huge;
  __device__ void operator()(int64_t v, int64_t e, int64_t x) const {
    const int32_t pos = (int32_t)(e & 0xffffffffLL);
    if (x & 1) out[pos] = (int32_t)v;
    if (x >> 32) huge[e >> 32] = pos;
  }
};

__global__ void k_level_stats(int32_t n, const int64_t* __restrict__ xadj, const int32_t* __restrict__ vw,
                              int32_t mid_deg, unsigned long long* out) {
  unsigned long long mhi = 0, mdeg = 0, mvw = 0, mhuge = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = (unsigned long long)(xadj[v + 1] - xadj[v]);
    if (d > (unsigned long long)kLowDeg) mhi += d;
    if (d > (unsigned long long)mid_deg) mhuge += d;
    mdeg = d > mdeg ? d : mdeg;
    const unsigned long long w = (unsigned long long)vw[v];
    mvw = w > mvw ? w : mvw;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mhi += __shfl_xor_sync(0xffffffffu, mhi, o);
    mhuge += __shfl_xor_sync(0xffffffffu, mhuge, o);
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mdeg, o);
    mdeg = y > mdeg ? y : mdeg;
    const unsigned long long z = __shfl_xor_sync(0xffffffffu, mvw, o);
    mvw = z > mvw ? z : mvw;
  }
  if ((threadIdx.x & 31) == 0) {
    if (mhi) atomicAdd(&out[0], mhi);
    if (mdeg) atomicMax(&out[1], mdeg);
    if (mvw) atomicMax(&out[2], mvw);
    if (mhuge) atomicAdd(&out[3], mhuge);
  }
}
}  // namespace

namespace {
// Chunk map of the flattened hub entries: chunk c starts in the row r with
// pre[r] <= c * kHubChunk < pre[r + 1].
__global__ void k_hub_chunks(int32_t n_huge, const int64_t* __restrict__ pre, int32_t* chunk) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_huge; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c0 = (pre[r] + kHubChunk - 1) / kHubChunk, c1 = (pre[r + 1] + kHubChunk - 1) / kHubChunk;
    for (int64_t c = c0; c < c1; c++) chunk[c] = (int32_t)r;
  }
}

struct LoadSplit {
  const int32_t* hi;
  const int32_t* huge;
  const int64_t* xadj;
  int64_t split_deg;
  __device__ int64_t operator()(int64_t j) const {
    const int32_t v = hi[huge[j]];
    return xadj[v + 1] - xadj[v] > split_deg ? 1 : 0;
  }
};
struct StoreSplit {
  int32_t* sidx;
  int32_t* list;
  __device__ void operator()(int64_t j, int64_t e, int64_t x) const {
    sidx[j] = x ? (int32_t)e : -1;
    if (x) list[e] = (int32_t)j;
  }
};

struct LoadHubDeg {
  const int32_t* hi;
  const int32_t* huge;
  const int64_t* xadj;
  __device__ int64_t operator()(int64_t j) const {
    const int32_t v = hi[huge[j]];
    return xadj[v + 1] - xadj[v];
  }
};

// one device value read back through the context's pinned block (slot 5)
int64_t read_i64_at(Ctx& c, const int64_t* d) {
  GM_CUDA(cudaMemcpyAsync(c.h_small + 5, d, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  return c.h_small[5];
}

// The flattened entries of the rows of degree > mid_deg (in huge[] order)
// and their chunk map, so that kernels can spread those rows over CTAs;
// rows above split_deg sum per-chunk PE tables.
void prepare_hubs(Ctx& c, Level& L, int64_t split_deg) {
  if (!L.n_huge) {
    L.n_hub_chunks = 0;
    return;
  }
  if (!L.hub_pre) L.hub_pre = c.mem.make<int64_t>((size_t)L.n + 1);
  const int64_t nch = (L.m_huge + kHubChunk - 1) / kHubChunk;
  if (!L.hub_chunk || L.hub_chunk_cap < nch + 1) {
    // captured graphs hold the old pointers
    drop_graph(L);
    if (L.cgexec) cudaGraphExecDestroy(L.cgexec);
    L.cgexec = nullptr;
    if (L.hub_chunk) c.mem.put(L.hub_chunk);
    if (L.hub_part) c.mem.put(L.hub_part);
    L.hub_chunk_cap = nch + 1;
    L.hub_chunk = c.mem.make<int32_t>((size_t)L.hub_chunk_cap);
    L.hub_part = c.mem.make<unsigned long long>((size_t)L.hub_chunk_cap * 4);
  }
  scan(LoadHubDeg{L.hi, L.huge, L.xadj}, StoreExcl{L.hub_pre}, L.n_huge, nullptr, c.scan, c.st);
  const int64_t tiles = std::max<int64_t>(1, scan_tiles(L.n_huge));
  GM_CUDA(cudaMemcpyAsync(L.hub_pre + L.n_huge, c.scan.tile_sums + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                          c.st));
  k_hub_chunks<<<grid_for(c, kThreads, L.n_huge), kThreads, 0, c.st>>>(L.n_huge, L.hub_pre, L.hub_chunk);
  count_launch();
  L.n_hub_chunks = nch;
  if (!L.hub_acc) {
    L.hub_acc = c.mem.make<int64_t>((size_t)std::max(1, L.n));
    GM_CUDA(cudaMemsetAsync(L.hub_acc, 0, (size_t)std::max(1, L.n) * sizeof(int64_t), c.st));
  }
  // the rows whose PE-code tables are summed over chunks
  if (!L.hub_sidx) L.hub_sidx = c.mem.make<int32_t>((size_t)std::max(1, L.n));
  if (!L.hub_split) L.hub_split = c.mem.make<int32_t>((size_t)std::max(1, L.n));
  scan(LoadSplit{L.hi, L.huge, L.xadj, split_deg}, StoreSplit{L.hub_sidx, L.hub_split}, L.n_huge, nullptr, c.scan,
       c.st);
  int64_t ns = read_i64_at(c, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(L.n_huge)));
  const int64_t need = ns * c.topo.kc;
  if (need * (int64_t)sizeof(int32_t) > kSplitTableBytes) {
    ns = 0;  // too many: every row is rated whole
    L.hub_split_deg = INT64_MAX;
  } else {
    L.hub_split_deg = split_deg;
  }
  L.n_split = (int32_t)ns;
  if (ns && L.hub_gtab_cap < need) {
    drop_graph(L);
    if (L.hub_gtab) c.mem.put(L.hub_gtab);
    L.hub_gtab_cap = need;
    L.hub_gtab = c.mem.make<int32_t>((size_t)need);
    GM_CUDA(cudaMemsetAsync(L.hub_gtab, 0, (size_t)need * sizeof(int32_t), c.st));
  }
}
}  // namespace

// Degree classes of a level with the warp-per-vertex bound mid_deg and the
// hub split bound split_deg.
void classify_with(Ctx& c, Level& L, int32_t mid_deg, int64_t split_deg) {
  if (!L.hi) L.hi = c.mem.make<int32_t>((size_t)std::max(1, L.n));
  if (!L.huge) L.huge = c.mem.make<int32_t>((size_t)std::max(1, L.n));
  L.mid_deg = mid_deg;
  scan(LoadHigh{L.xadj, mid_deg}, StoreHigh{L.hi, L.huge}, L.n, nullptr, c.scan, c.st);
  unsigned long long* st = reinterpret_cast<unsigned long long*>(c.d_stats);
  GM_CUDA(cudaMemsetAsync(st, 0, 4 * sizeof(int64_t), c.st));
  const int64_t blocks = std::min<int64_t>(((int64_t)L.n + 255) / 256, (int64_t)c.num_sms * 8);
  k_level_stats<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, c.st>>>(L.n, L.xadj, L.vw, mid_deg, st);
  count_launch();
  // count of high-degree vertices and the four statistics, one synchronisation
  GM_CUDA(cudaMemcpyAsync(c.h_small, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(L.n)), sizeof(int64_t),
                          cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(c.h_small + 1, st, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  L.n_hi = (int32_t)(c.h_small[0] & 0xffffffffLL);
  L.n_huge = (int32_t)(c.h_small[0] >> 32);
  L.m_hi = c.h_small[1];
  L.max_deg = c.h_small[2];
  L.max_vw = (int32_t)c.h_small[3];
  L.m_huge = c.h_small[4];
  prepare_hubs(c, L, split_deg);
}

namespace {
// The schedule autotuner.  A level whose rows of degree > kLowDeg hold at
// least kTuneMinEntries entries gets its warp-per-vertex bound mid_deg
// (candidates 255, 128, 64: which rows a warp takes and which the hub
// kernels) and its hub split bound (candidates 4096, 2048, 16384: which hub
// rows one CTA rates whole and which sum per-chunk tables) chosen by timing a
// probe, coordinate by coordinate; the choice is cached per (device, n, m,
// entries of degree > kLowDeg, largest degree, PE code space) for the
// process.  Every schedule gives the same result; only the time differs.
constexpr int64_t kTuneMinEntries = 1 << 20;
double now_wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
struct SchedKey {
  int dev;
  int32_t n;
  int64_t m, m_hi, max_deg;
  int32_t kc;
  bool operator==(const SchedKey& o) const {
    return dev == o.dev && n == o.n && m == o.m && m_hi == o.m_hi && max_deg == o.max_deg && kc == o.kc;
  }
};
struct SchedChoice {
  int32_t mid_deg;
  int64_t split_deg;
};
std::mutex g_sched_mutex;
std::vector<std::pair<SchedKey, SchedChoice>> g_sched_cache;

// Device time of the probe, best of two: a full J evaluation and Alg. 4
// step 1 over the vertices of degree > kLowDeg (per-warp and hub tables),
// with no vertex locked and the outputs in transient scratch (the
// rebalancing buffers), on the level's mapping, which is zeroed first on a
// coarse level (it is set later by projection or the initial mapping).
double probe_ms(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  struct ProfOff {  // the probe's launches stay out of the kernel-class profile
    Ctx& c;
    bool was;
    explicit ProfOff(Ctx& cc) : c(cc), was(cc.prof) { cc.prof = false; }
    ~ProfOff() { c.prof = was; }
  } prof_off(c);
  if (lvl > 0) GM_CUDA(cudaMemsetAsync(L.pi, 0, (size_t)std::max(1, L.n) * sizeof(int32_t), c.st));
  GM_CUDA(cudaMemsetAsync(c.sel, 0, (size_t)std::max(1, L.n), c.st));
  const GroupLayout glay = group_layout(c.topo);
  const LpFilter flt{0, 1};
  cudaEvent_t e0, e1;
  GM_CUDA(cudaEventCreate(&e0));
  GM_CUDA(cudaEventCreate(&e1));
  double best = 1e30;
  for (int rep = 0; rep < 2; rep++) {
    GM_CUDA(cudaEventRecord(e0, c.st));
    launch_eval(c, lvl, nullptr, true);
    if (L.n_hi > L.n_huge) {
      const size_t sm = mid_table_smem(glay.total);
      k_lp_gain_mid<<<mid_grid(c, (const void*)k_lp_gain_mid, sm, L.n_hi), kMidThreads, sm, c.st>>>(
          view(L), L.hi, L.n_hi, L.pi, c.sel, c.dest, c.P64, c.elig, c.topo, glay, flt, c.probe_state);
      count_launch();
    }
    if (L.n_huge) {
      const LpHubPolicy pol{L.pi, c.sel, c.dest, c.P64, c.elig, c.topo, glay, flt, c.probe_state};
      launch_hub_tab(c, L, pol, (size_t)glay.total * sizeof(int32_t));
    }
    GM_CUDA(cudaEventRecord(e1, c.st));
    GM_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}
}  // namespace

void classify_degrees(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  const int32_t prev_mid = L.mid_deg;
  const int64_t prev_split = L.split_req;
  const bool fixed = c.cfg.mid_deg > 0 || c.cfg.split_deg > 0;
  SchedChoice ch{c.cfg.mid_deg > 0 ? c.cfg.mid_deg : kMidDeg, c.cfg.split_deg > 0 ? c.cfg.split_deg : kSplitDeg};
  classify_with(c, L, ch.mid_deg, ch.split_deg);
  L.tuned = 0;
  if (!fixed && L.m_hi >= kTuneMinEntries && mid_tables(c)) {
    const SchedKey key{c.dev, L.n, L.m, L.m_hi, L.max_deg, c.topo.kc};
    bool hit = false;
    {
      std::lock_guard<std::mutex> lock(g_sched_mutex);
      for (const auto& kv : g_sched_cache)
        if (kv.first == key) {
          ch = kv.second;
          hit = true;
        }
    }
    if (!hit) {
      const double t0 = now_wall_ms();
      double best = probe_ms(c, lvl);
      SchedChoice cur = ch;
      for (int32_t md : {128, 64}) {
        classify_with(c, L, md, cur.split_deg);
        const double t = probe_ms(c, lvl);
        if (t < best) {
          best = t;
          ch = SchedChoice{md, cur.split_deg};
        }
      }
      cur = ch;
      for (int64_t sd : {(int64_t)2048, (int64_t)16384}) {
        classify_with(c, L, cur.mid_deg, sd);
        const double t = probe_ms(c, lvl);
        if (t < best) {
          best = t;
          ch = SchedChoice{cur.mid_deg, sd};
        }
      }
      c.ms_tune += now_wall_ms() - t0;
      std::lock_guard<std::mutex> lock(g_sched_mutex);
      g_sched_cache.emplace_back(key, ch);
    }
    classify_with(c, L, ch.mid_deg, ch.split_deg);
    L.tuned = 1;
  }
  L.split_req = ch.split_deg;
  if (L.mid_deg != prev_mid || L.split_req != prev_split) {
    // kernels captured for the other schedule
    drop_graph(L);
    if (L.cgexec) cudaGraphExecDestroy(L.cgexec);
    L.cgexec = nullptr;
  }
}

}  // namespace gm
