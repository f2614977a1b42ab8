// Coarsening engine: graph validation, label-propagation clustering,
// contraction by sort + segmented reduce, projection (uncontraction) and the
// initial mapping of the coarsest graph.
//
// Clustering (the clustering alternative named in Sections 2.1 and 4.2):
// clusters start as singletons; in each of two sub-rounds per iteration the
// active half of the vertices (a hash bit) rates the neighbouring clusters by
// edge weight (own cluster included), ties to the smaller tie-hash, then the
// smaller label; requests into a cluster are admitted in (hash, id) order
// while it stays within the weight cap.  Only over-subscribed clusters need
// that order, so only their requests are sorted.  Every decision is a
// function of values, never of thread timing, which keeps the result
// bit-identical to a serial evaluation.
//
// Contraction (Section 2.1 semantics, replacing the CAS hashing of Alg. 3):
// keys (M(u), M(v)) of the non-self-loop edges are radix-sorted, equal keys
// are reduced by a prefix sum of the weights, and the coarse CSR rows follow
// from the sorted unique keys, so adjacency order is deterministic.
#include <algorithm>
#include <atomic>
#include <chrono>

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

// Persistent grid of a warp-tile kernel: one wave of resident blocks.
inline unsigned tile_grid(Ctx& c, const void* fn, int64_t n) {
  const int64_t tiles = (n + kTileV - 1) / kTileV;
  int64_t g = (tiles + kTileWarps - 1) / kTileWarps;
  const int64_t cap = (int64_t)c.num_sms * c.resident_blocks(fn, kTileThreads, 0);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Grid of a mid-degree kernel (one warp per vertex of the high-degree list).
inline unsigned mid_grid(Ctx& c, const void* fn, size_t smem, int64_t n_hi) {
  int64_t g = (n_hi + kMidWarps - 1) / kMidWarps;
  const int64_t cap = (int64_t)c.num_sms * c.resident_blocks(fn, kMidThreads, smem);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

inline unsigned grid_for(const Ctx& c, int64_t items_per_block, int64_t n) {
  int64_t g = (n + items_per_block - 1) / items_per_block;
  int64_t cap = (int64_t)c.num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------
// validation of the input graph
// ---------------------------------------------------------------------------
// Input validation, pass 1, one thread per vertex: row bounds (monotone
// xadj within [0, m]) and vertex weights.
__global__ void __launch_bounds__(kThreads) k_validate_rows(GraphView g, int64_t m, uint32_t* err,
                                                           unsigned long long* sums) {
  uint32_t e_local = 0;
  unsigned long long sv = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t beg = g.xadj[v], end = g.xadj[v + 1];
    if (beg < 0 || end < beg || end > m) e_local |= ERR_XADJ;
    if (g.vw[v] < 1) e_local |= ERR_WEIGHT;
    else sv += (unsigned long long)g.vw[v];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e_local |= __shfl_xor_sync(0xffffffffu, e_local, o);
    sv += __shfl_xor_sync(0xffffffffu, sv, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e_local) atomicOr(err, e_local);
    if (sv) atomicAdd(&sums[0], sv);
  }
}

// Pass 2 (rows known valid), every thread a run of kValChunk consecutive CSR
// entries, so that rows of any length spread evenly: range, self-loop,
// strictly ascending rows, weights, and the reverse entry with the same
// weight (binary search in the neighbour's row).
constexpr int64_t kValChunk = 64;
__global__ void __launch_bounds__(kThreads) k_validate_entries(GraphView g, int64_t m, uint32_t* err,
                                                              unsigned long long* sums) {
  uint32_t e_local = 0;
  unsigned long long sw = 0, n_search = 0, n_other = 0;
  const int64_t chunks = (m + kValChunk - 1) / kValChunk;
  for (int64_t ch = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ch < chunks;
       ch += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = ch * kValChunk, e1 = min(m, e0 + kValChunk);
    int64_t lo = 0, hi = g.n;  // the row holding e0: xadj[lo] <= e0 < xadj[hi]
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (g.xadj[mid] <= e0) lo = mid;
      else hi = mid;
    }
    int64_t v = lo;
    for (int64_t e = e0; e < e1; e++) {
      while (v < g.n - 1 && g.xadj[v + 1] <= e) v++;
      const int64_t beg = g.xadj[v];
      const int32_t u = g.adj[e];
      const int32_t w = g.adjw[e];
      if (u < 0 || u >= g.n) {
        e_local |= ERR_RANGE;
        continue;
      }
      if (u == v) e_local |= ERR_SELFLOOP;
      if (e > beg && g.adj[e - 1] >= u) e_local |= ERR_UNSORTED;
      if (w < 1) e_local |= ERR_WEIGHT;
      else sw += (unsigned long long)w;
      if (u == v) continue;
      // symmetry: the entry looks for its twin (u, v) only when row u is the
      // smaller of the two rows (by degree, then id), so every search runs in
      // the shorter row; the others are counted.  Rows being strictly
      // ascending, the twin map from the searching entries to the others is
      // injective, so equal counts (checked on the host) make it a bijection.
      const int64_t ub = g.xadj[u], ue = g.xadj[u + 1];
      const int64_t du = ue - ub, dv = g.xadj[v + 1] - beg;
      if (!(du < dv || (du == dv && u < v))) {
        n_other++;
        continue;
      }
      n_search++;
      int64_t l = ub, r = ue;
      while (l < r) {  // first entry >= v in row u
        const int64_t mid = (l + r) >> 1;
        if (g.adj[mid] < v) l = mid + 1;
        else r = mid;
      }
      if (l >= ue || g.adj[l] != (int32_t)v || g.adjw[l] != w) e_local |= ERR_ASYM;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e_local |= __shfl_xor_sync(0xffffffffu, e_local, o);
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    n_search += __shfl_xor_sync(0xffffffffu, n_search, o);
    n_other += __shfl_xor_sync(0xffffffffu, n_other, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e_local) atomicOr(err, e_local);
    if (sw) atomicAdd(&sums[1], sw);
    if (n_search) atomicAdd(&sums[2], n_search);
    if (n_other) atomicAdd(&sums[3], n_other);
  }
}

__global__ void k_iota(int32_t* a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// clustering
// ---------------------------------------------------------------------------
struct ClusterArgs {
  const int32_t* C;      // labels (snapshot)
  const int32_t* Wc;     // cluster weights (snapshot)
  int32_t* ReqW;         // requested weight per target
  int32_t* req;          // requested target per vertex (-1 none)
  int64_t wcap;
  uint64_t seed;
  const ClusterState* cs;  // current iteration
  int32_t level;
  int32_t round;
};

__device__ __forceinline__ bool cluster_active(const ClusterArgs& a, int32_t v, int64_t deg) {
  return deg > 0 && (int32_t)((h_active(a.seed, a.level, v) >> a.cs->it) & 1ULL) == a.round;
}

__device__ __forceinline__ void cluster_request(const ClusterArgs& a, int32_t v, int32_t own, int32_t best,
                                                int32_t cv) {
  if (best != own && (int64_t)a.Wc[best] + cv <= a.wcap) {
    a.req[v] = best;
    atomicAdd(&a.ReqW[best], cv);
  } else {
    a.req[v] = -1;
  }
}

struct GatherLabel {
  const int32_t* __restrict__ C;
  __device__ __forceinline__ int32_t operator()(int32_t u) const { return C[u]; }
};

// Clustering ratings for the low-degree vertices.  Warp tiles stage the
// neighbour labels; the active vertices of a tile are then rated four at a
// time by 8-lane sub-warps reading the staged entries from shared memory.
// In a tile whose CSR range exceeds the staging capacity (a high-degree row
// inside, as on power-law graphs) each sub-warp first copies its vertex's
// row (at most kLowDeg entries) into its quarter of the warp's buffer.
static_assert(kTileE / 4 >= kLowDeg, "a sub-warp's quarter of the staging buffer holds one low-degree row");
__global__ void __launch_bounds__(kTileThreads, 9) k_cluster_tile(GraphView g, ClusterArgs a) {
  __shared__ int2 scw[kTileWarps][kTileE];  // (label, weight) per staged entry
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane >> 3, sl = lane & 7;
  const TileGraph tg{g.n, g.xadj, g.adj, g.adjw};
  const int64_t ntiles = ((int64_t)g.n + kTileV - 1) / kTileV;
  for (int64_t tile = (int64_t)blockIdx.x * kTileWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kTileWarps) {
    const TileLane t = stage_tile_packed(tg, tile * kTileV, lane, scw[warp], GatherLabel{a.C});
    const int deg = (int)(t.e - t.b);
    const bool low = t.v < g.n && deg <= kLowDeg;
    const bool active = low && cluster_active(a, (int32_t)t.v, deg);
    int32_t own = active ? a.C[t.v] : -1;
    if (low && !active) a.req[t.v] = -1;
    const unsigned work = __ballot_sync(0xffffffffu, active);
    const int rank = __popc(work & ((1u << lane) - 1u));
    const int rounds = (__popc(work) + 3) / 4;
    for (int r = 0; r < rounds; r++) {
      const int src = tile_worker_ranked(work, rank, r, sub, lane);
      const int s2 = src < 0 ? 0 : src;
      const int64_t vb = __shfl_sync(0xffffffffu, t.b, s2);
      int off = (int)(vb - t.E0);
      const int dg = (int)(__shfl_sync(0xffffffffu, t.e, s2) - vb);
      const int32_t ow = __shfl_sync(0xffffffffu, own, s2);
      if (!t.staged) {  // warp-uniform
        off = sub * (kTileE / 4);
        __syncwarp();  // the previous round has read this quarter
        if (src >= 0)
          for (int j = sl; j < dg; j += kSubWarp) scw[warp][off + j] = make_int2(a.C[g.adj[vb + j]], g.adjw[vb + j]);
        __syncwarp();
      }
      const int2* cw = scw[warp] + off;
      // best (score, tie-hash, label) over this lane's candidates; the hash
      // of the current best is computed once, on the first tie
      int32_t bs = 0, bt = -1, so = 0;
      uint64_t bh = 0;
      bool bhk = false;
      if (src >= 0) {
        for (int j = sl; j < dg; j += kSubWarp) {
          const int2 xj = cw[j];
          const int32_t cj = xj.x;
          so += (cj == ow) ? xj.y : 0;
          if (cj == ow || cj == bt) continue;
          int32_t scj = 0;
#pragma unroll 4
          for (int l = 0; l < dg; l++) {
            const int2 x = cw[l];
            scj += (x.x == cj) ? x.y : 0;
          }
          if (bt < 0 || scj > bs) {
            bs = scj;
            bt = cj;
            bhk = false;
            continue;
          }
          if (scj < bs) continue;
          if (!bhk) {
            bh = h_tie(a.seed, a.level, bt);
            bhk = true;
          }
          const uint64_t hj = h_tie(a.seed, a.level, cj);
          if (hj < bh || (hj == bh && cj < bt)) {
            bt = cj;
            bh = hj;
          }
        }
      }
      if (bt >= 0 && !bhk) bh = h_tie(a.seed, a.level, bt);
#pragma unroll
      for (int o = kSubWarp / 2; o > 0; o >>= 1) {
        so += __shfl_xor_sync(0xffffffffu, so, o);
        const int32_t os = __shfl_xor_sync(0xffffffffu, bs, o);
        const int32_t ot = __shfl_xor_sync(0xffffffffu, bt, o);
        const uint64_t oh = __shfl_xor_sync(0xffffffffu, bh, o);
        if (ot >= 0 && (bt < 0 || os > bs || (os == bs && (oh < bh || (oh == bh && ot < bt))))) {
          bs = os;
          bt = ot;
          bh = oh;
        }
      }
      if (src >= 0 && sl == 0) {
        const int32_t v = (int32_t)(tile * kTileV + src);
        // against the own cluster: larger score, then smaller tie-hash, then smaller label
        bool take = bt >= 0 && bs >= so;
        if (take && bs == so) {
          const uint64_t ho = h_tie(a.seed, a.level, ow);
          take = bh < ho || (bh == ho && bt < ow);
        }
        cluster_request(a, v, ow, take ? bt : ow, g.vw[v]);
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ uint32_t slot_hash(int32_t t) {
  uint32_t x = (uint32_t)t * 0x9E3779B1u;
  return x ^ (x >> 15);
}

// Vertices of degree > kMidDeg (up to 1.6e5 entries on R-MAT scale 22).
// Each row is rated in an open-addressing table (next power of two >= 2
// (deg + 1) slots, at least 64, linear probing) of 64-bit words, (label <<
// 32) | summed weight: a new label costs one compare-and-swap, a repeated one
// a compare-and-swap and an add (the weight sum of a row stays below 2^31, so
// it never carries into the label).  The own cluster is inserted with weight
// 0.  The decision takes the largest weight, then the smaller tie-hash, then
// the smaller label, and puts every slot back to empty.
//  * rows of at most kSmemRowDeg entries: the whole row on one CTA, its
//    table in shared memory (no global atomics);
//  * larger rows: their entries, flattened in huge[] order, are cut into
//    chunks of kHubChunk entries that the CTAs of one wave take in turn, the
//    table in global memory.  A second launch reads the table back in the
//    same chunks (each chunk takes the slots in proportion to its share of
//    the row's entries) and stores each slice's best label; a third combines
//    the slices of every row and files its request.
constexpr unsigned long long kEmptySlot = ~0ULL;
constexpr int64_t kSmemRowDeg = 2047;
constexpr uint32_t kSmemSlots = 4096;  // >= 2 (kSmemRowDeg + 1)
static_assert(kSmemSlots >= 2 * (kSmemRowDeg + 1), "shared-memory row table at most half full");
// rows of one chunk at most: every row there has more than kLowDeg + 1 >= 33 entries
constexpr int kChunkRows = 64;
// rows of at most kGroupRowDeg entries are rated by kRowGroups thread groups
// of a CTA side by side, each with its share of the shared-memory table
constexpr int kRowGroups = 2;
constexpr int64_t kGroupRowDeg = kSmemSlots / kRowGroups / 2 - 1;
static_assert(kSmemSlots / kRowGroups >= 2 * (kGroupRowDeg + 1), "a group's table at most half full");
static_assert(kRowGroups <= 2, "named barriers 1 and 2 serve the row groups");
static_assert(kHubChunk / 34 + 2 <= kChunkRows, "a chunk's rows fit the per-chunk row table");

// Inserts from slot h on (`probes` already made).
__device__ __forceinline__ bool hub_insert_from(unsigned long long* T, uint32_t mask, int32_t t, int32_t w, uint32_t h,
                                                uint32_t probes) {
  const unsigned long long key = (unsigned long long)(uint32_t)t << 32;
  for (uint32_t probe = probes; probe <= mask; probe++) {
    const unsigned long long prev = atomicCAS(&T[h], kEmptySlot, key | (uint32_t)w);
    if (prev == kEmptySlot) return true;
    if ((prev >> 32) == (uint32_t)t) {
      if (w) atomicAdd(&T[h], (unsigned long long)(uint32_t)w);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}
__device__ __forceinline__ bool hub_insert(unsigned long long* T, uint32_t mask, int32_t t, int32_t w) {
  return hub_insert_from(T, mask, t, w, slot_hash(t) & mask, 0);
}

// entries a thread keeps in flight
constexpr int kHubBatch = 4;

// The threads that rate one row together: the whole CTA (barrier 0), or one
// of the groups of consecutive warps that rate rows side by side, each with
// its own named barrier.
struct RowGroup {
  int tid, size;    // thread index in the group, group size (a multiple of 32)
  int warp0, warps; // the group's warps within the CTA
  int bar;          // 0: the CTA barrier; else a named barrier of `size` threads
  __device__ __forceinline__ void sync() const {  // (immediate barrier ids: the kernel reserves three)
    if (bar == 0) __syncthreads();
    else if (bar == 1) asm volatile("bar.sync 1, %0;" ::"r"(size) : "memory");
    else asm volatile("bar.sync 2, %0;" ::"r"(size) : "memory");
  }
};
__device__ __forceinline__ RowGroup cta_group() {
  return RowGroup{(int)threadIdx.x, (int)blockDim.x, 0, (int)(blockDim.x >> 5), 0};
}

// Inserts the CSR entries [e0, e1) of a row (labels gathered from C) by the
// threads of group gr: per thread kHubBatch entries at a time, whose loads,
// label gathers and first compare-and-swaps are each issued before any
// result is used; only collisions with another label probe on.  Returns
// false if a table overflowed.
__device__ __forceinline__ bool hub_insert_range(const GraphView& g, const int32_t* __restrict__ C, int64_t e0,
                                                 int64_t e1, unsigned long long* T, uint32_t mask,
                                                 const RowGroup& gr) {
  bool ok = true;
  for (int64_t f0 = e0; f0 < e1; f0 += (int64_t)gr.size * kHubBatch) {
    int32_t t[kHubBatch], w[kHubBatch];
    uint32_t h[kHubBatch];
    unsigned long long prev[kHubBatch];
#pragma unroll
    for (int b = 0; b < kHubBatch; b++) {
      const int64_t e = f0 + (int64_t)b * gr.size + gr.tid;
      t[b] = e < e1 ? g.adj[e] : -1;
      w[b] = e < e1 ? g.adjw[e] : 0;
    }
#pragma unroll
    for (int b = 0; b < kHubBatch; b++) t[b] = t[b] >= 0 ? C[t[b]] : -1;
#pragma unroll
    for (int b = 0; b < kHubBatch; b++) {
      h[b] = slot_hash(t[b]) & mask;
      prev[b] = t[b] >= 0 ? atomicCAS(&T[h[b]], kEmptySlot, ((unsigned long long)(uint32_t)t[b] << 32) | (uint32_t)w[b])
                          : kEmptySlot;
    }
#pragma unroll
    for (int b = 0; b < kHubBatch; b++) {
      if (t[b] < 0 || prev[b] == kEmptySlot) continue;
      if ((prev[b] >> 32) == (uint32_t)t[b]) {
        if (w[b]) atomicAdd(&T[h[b]], (unsigned long long)(uint32_t)w[b]);
      } else {
        ok &= hub_insert_from(T, mask, t[b], w[b], (h[b] + 1) & mask, 1);
      }
    }
  }
  return ok;
}

struct HubScratch {
  int32_t bs[kHiThreads / 32];
  uint64_t bh[kHiThreads / 32];
  int32_t bt[kHiThreads / 32];
};

// The best label of the slots T[s0, s1) of a row table (kGlobal: read from
// L2, where other CTAs' atomics were performed): the largest weight, then
// the smaller tie-hash, then the smaller label, in two passes so that only
// labels of the largest weight are hashed; every slot is put back to empty.
// All threads of group gr call it; the group's thread 0 receives the result
// (bs = -1 for no label); ends with the group's barrier.
template <bool kGlobal>
__device__ __forceinline__ void table_best(unsigned long long* T, uint32_t s0, uint32_t s1, const ClusterArgs& a,
                                           HubScratch& sx, const RowGroup& gr, int32_t& out_bs, uint64_t& out_bh,
                                           int32_t& out_bt) {
  const int warp = (int)(threadIdx.x >> 5);
  int32_t bs = -1;
#pragma unroll 4
  for (uint32_t s = s0 + gr.tid; s < s1; s += gr.size) {
    const unsigned long long x = kGlobal ? __ldcg(T + s) : T[s];
    if (x != kEmptySlot) bs = max(bs, (int32_t)(uint32_t)x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bs = max(bs, __shfl_xor_sync(0xffffffffu, bs, o));
  if ((threadIdx.x & 31) == 0) sx.bs[warp] = bs;
  gr.sync();
  bs = sx.bs[gr.warp0];
  for (int w = 1; w < gr.warps; w++) bs = max(bs, sx.bs[gr.warp0 + w]);
  uint64_t bh = ~0ULL;
  int32_t bt = INT32_MAX;
#pragma unroll 4
  for (uint32_t s = s0 + gr.tid; s < s1; s += gr.size) {
    const unsigned long long x = kGlobal ? __ldcg(T + s) : T[s];
    if (x == kEmptySlot) continue;
    T[s] = kEmptySlot;
    if ((int32_t)(uint32_t)x != bs) continue;
    const int32_t t = (int32_t)(x >> 32);
    const uint64_t h = h_tie(a.seed, a.level, t);
    if (h < bh || (h == bh && t < bt)) {
      bh = h;
      bt = t;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t oh = __shfl_xor_sync(0xffffffffu, bh, o);
    const int32_t ot = __shfl_xor_sync(0xffffffffu, bt, o);
    if (oh < bh || (oh == bh && ot < bt)) {
      bh = oh;
      bt = ot;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sx.bh[warp] = bh;
    sx.bt[warp] = bt;
  }
  gr.sync();
  if (gr.tid == 0) {
    for (int w = 1; w < gr.warps; w++) {
      const uint64_t h = sx.bh[gr.warp0 + w];
      const int32_t t = sx.bt[gr.warp0 + w];
      if (h < bh || (h == bh && t < bt)) {
        bh = h;
        bt = t;
      }
    }
    out_bs = bs;
    out_bh = bh;
    out_bt = bt;
  }
  gr.sync();
}

// The larger rows' slice results: per chunk two slots (0: the large row
// holding the chunk's first entry, 1: a large row starting inside the chunk;
// a row of at least kSmemRowDeg + 1 >= kHubChunk entries leaves room for no
// other), each ((weight << 32) | label, tie-hash).
__device__ __forceinline__ int64_t part_slot(int64_t ch, int64_t rb) {
  return 4 * ch + (rb >= ch * kHubChunk ? 2 : 0);
}

// Sub-round step 1 for the rows of degree > kMidDeg: the rows on the
// shared-memory path are rated and decided here; the larger rows only insert.
__global__ void __launch_bounds__(kHiThreads, 5) k_cluster_high(GraphView g, HubRows hr,
                                                             const int64_t* __restrict__ hoff,
                                                             unsigned long long* htab, ClusterArgs a,
                                                             unsigned long long* ctr, uint32_t* err) {
  static_assert(kHiThreads >= kChunkRows, "one thread per row of a chunk");
  static_assert(kHiThreads % (32 * kRowGroups) == 0, "whole warps per row group");
  __shared__ unsigned long long stab[kSmemSlots];  // the groups' tables side by side, or one CTA table
  __shared__ HubScratch sx;
  __shared__ int32_t s_bs[kRowGroups], s_bt[kRowGroups];
  __shared__ uint64_t s_bh[kRowGroups];
  __shared__ int64_t s_ch;
  // the rows of the current chunk, looked up at once (one thread each): a
  // row's lookup is a chain of dependent loads that would otherwise run
  // row after row
  __shared__ int32_t s_v[kChunkRows];  // -1: nothing for this chunk to do
  __shared__ int32_t s_own[kChunkRows], s_idx[kChunkRows];
  __shared__ int64_t s_rb[kChunkRows], s_re[kChunkRows], s_x0[kChunkRows];
  for (uint32_t s = threadIdx.x; s < kSmemSlots; s += blockDim.x) stab[s] = kEmptySlot;
  __syncthreads();
  const int64_t m_hub = hr.pre[hr.n_huge];
  for (int64_t ch = next_chunk(ctr, &s_ch); ch < hr.nchunks; ch = next_chunk(ctr, &s_ch)) {
    const int64_t cb = ch * kHubChunk, ce = min(cb + kHubChunk, m_hub);
    const int32_t r = hr.chunk[ch] + (int32_t)threadIdx.x;
    bool row = false;
    if (threadIdx.x < kChunkRows) {
      int32_t v = -1;
      int64_t rb = 0, re = 0;
      if (r < hr.n_huge) {
        rb = hr.pre[r];
        re = hr.pre[r + 1];
        row = rb < ce;
      }
      const int64_t deg = re - rb;
      const bool first = rb >= cb;  // this chunk holds the row's first entry
      // a row on the shared-memory path belongs to the chunk of its first entry
      if (row && (deg > kSmemRowDeg || first)) {
        const int32_t idx = hr.huge[r];
        const int32_t u = hr.hi[idx];
        if (cluster_active(a, u, deg)) {
          v = u;
          s_idx[threadIdx.x] = idx;
          s_own[threadIdx.x] = a.C[u];
          s_x0[threadIdx.x] = g.xadj[u] - rb;  // CSR position of flat entry f: x0 + f
        } else if (first) {
          a.req[u] = -1;
        }
      }
      s_v[threadIdx.x] = v;
      s_rb[threadIdx.x] = rb;
      s_re[threadIdx.x] = re;
    }
    const int nrows = __syncthreads_count(row);  // the chunk's rows are a prefix
    {
      // rows of at most kGroupRowDeg entries: the row groups side by side,
      // row i to group i mod kRowGroups, each with its part of the table
      constexpr int kG = kHiThreads / kRowGroups;
      const int gi = (int)threadIdx.x / kG;
      const RowGroup gr{(int)threadIdx.x % kG, kG, gi * (kG / 32), kG / 32, 1 + gi};
      unsigned long long* gtab = stab + gi * (kSmemSlots / kRowGroups);
      for (int i = gi; i < nrows; i += kRowGroups) {
        const int32_t v = s_v[i];
        const int64_t deg = s_re[i] - s_rb[i];
        if (v < 0 || deg > kGroupRowDeg) continue;
        const int32_t own = s_own[i];
        uint32_t size = 64;
        while (size < 2 * (uint32_t)(deg + 1)) size <<= 1;
        bool ok = true;
        if (gr.tid == 0) ok = hub_insert(gtab, size - 1, own, 0);
        ok &= hub_insert_range(g, a.C, s_x0[i] + s_rb[i], s_x0[i] + s_re[i], gtab, size - 1, gr);
        if (!ok) atomicOr(err, ERR_CAPACITY);
        gr.sync();
        table_best<false>(gtab, 0, size, a, sx, gr, s_bs[gi], s_bh[gi], s_bt[gi]);
        if (gr.tid == 0) cluster_request(a, v, own, s_bt[gi], g.vw[v]);
      }
    }
    __syncthreads();  // the groups' tables are empty again: the whole table is the CTA's
    const RowGroup cta = cta_group();
    for (int i = 0; i < nrows; i++) {
      const int32_t v = s_v[i];
      if (v < 0) continue;
      const int64_t rb = s_rb[i], re = s_re[i], deg = re - rb, x0 = s_x0[i];
      if (deg <= kGroupRowDeg) continue;  // rated by a row group above
      const int32_t own = s_own[i];
      bool ok = true;
      if (deg <= kSmemRowDeg) {
        uint32_t size = 64;
        while (size < 2 * (uint32_t)(deg + 1)) size <<= 1;
        if (threadIdx.x == 0) ok = hub_insert(stab, size - 1, own, 0);
        ok &= hub_insert_range(g, a.C, x0 + rb, x0 + re, stab, size - 1, cta);
        if (!ok) atomicOr(err, ERR_CAPACITY);
        __syncthreads();
        table_best<false>(stab, 0, size, a, sx, cta, s_bs[0], s_bh[0], s_bt[0]);
        if (threadIdx.x == 0) cluster_request(a, v, own, s_bt[0], g.vw[v]);
        continue;
      }
      const int32_t idx = s_idx[i];
      const int64_t base = hoff[idx];
      const uint32_t mask = (uint32_t)(hoff[idx + 1] - base) - 1u;
      unsigned long long* T = htab + base;
      if (rb >= cb && threadIdx.x == 0) ok = hub_insert(T, mask, own, 0);
      ok &= hub_insert_range(g, a.C, x0 + max(rb, cb), x0 + min(re, ce), T, mask, cta);
      if (!ok) atomicOr(err, ERR_CAPACITY);
    }
  }
  leave_chunks(ctr);
}

// Sub-round step 2: every chunk reads back its slice of each larger row it
// overlaps (slots [S (f0 - rb) / deg, S (f1 - rb) / deg) of the row's S
// slots for its entries [f0, f1)), empties it and stores the slice's best.
__global__ void __launch_bounds__(kHiThreads) k_cluster_giant(HubRows hr, const int64_t* __restrict__ hoff,
                                                              unsigned long long* htab, unsigned long long* part,
                                                              ClusterArgs a, unsigned long long* ctr) {
  __shared__ HubScratch sx;
  __shared__ int32_t s_bs, s_bt;
  __shared__ uint64_t s_bh;
  __shared__ int64_t s_ch;
  __shared__ int32_t s_idx[kChunkRows];  // the chunk's active larger rows (-1: none)
  __shared__ int64_t s_rb[kChunkRows], s_re[kChunkRows];
  const int64_t m_hub = hr.pre[hr.n_huge];
  for (int64_t ch = next_chunk(ctr, &s_ch); ch < hr.nchunks; ch = next_chunk(ctr, &s_ch)) {
    const int64_t cb = ch * kHubChunk, ce = min(cb + kHubChunk, m_hub);
    const int32_t r = hr.chunk[ch] + (int32_t)threadIdx.x;
    bool row = false;
    if (threadIdx.x < kChunkRows) {
      int32_t idx = -1;
      int64_t rb = 0, re = 0;
      if (r < hr.n_huge) {
        rb = hr.pre[r];
        re = hr.pre[r + 1];
        row = rb < ce;
      }
      if (row && re - rb > kSmemRowDeg) {
        const int32_t j = hr.huge[r];
        if (cluster_active(a, hr.hi[j], re - rb)) idx = j;
      }
      s_idx[threadIdx.x] = idx;
      s_rb[threadIdx.x] = rb;
      s_re[threadIdx.x] = re;
    }
    const int nrows = __syncthreads_count(row);  // the chunk's rows are a prefix
    for (int i = 0; i < nrows; i++) {
      const int32_t idx = s_idx[i];
      if (idx < 0) continue;
      const int64_t rb = s_rb[i], re = s_re[i], deg = re - rb;
      const int64_t base = hoff[idx];
      const int64_t S = hoff[idx + 1] - base;
      const uint32_t s0 = (uint32_t)(S * (max(rb, cb) - rb) / deg), s1 = (uint32_t)(S * (min(re, ce) - rb) / deg);
      table_best<true>(htab + base, s0, s1, a, sx, cta_group(), s_bs, s_bh, s_bt);
      if (threadIdx.x == 0) {
        const int64_t p = part_slot(ch, rb);
        part[p] = ((unsigned long long)(uint32_t)s_bs << 32) | (uint32_t)s_bt;
        part[p + 1] = s_bh;
      }
    }
  }
  leave_chunks(ctr);
}

// Sub-round step 3: per active larger row (one thread each), the best of its
// slices, then its request.
__global__ void k_cluster_giant_finish(HubRows hr, const unsigned long long* __restrict__ part, const int32_t* vw,
                                       ClusterArgs a) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < hr.n_huge; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rb = hr.pre[r], re = hr.pre[r + 1];
    if (re - rb <= kSmemRowDeg) continue;
    const int32_t v = hr.hi[hr.huge[r]];
    if (!cluster_active(a, v, re - rb)) continue;
    int32_t bs = -1, bt = INT32_MAX;
    uint64_t bh = ~0ULL;
    for (int64_t ch = rb / kHubChunk; ch <= (re - 1) / kHubChunk; ch++) {
      const int64_t p = part_slot(ch, rb);
      const int32_t s = (int32_t)(part[p] >> 32), t = (int32_t)(uint32_t)part[p];
      const uint64_t h = part[p + 1];
      if (s > bs || (s == bs && (h < bh || (h == bh && t < bt)))) {
        bs = s;
        bt = t;
        bh = h;
      }
    }
    cluster_request(a, v, a.C[v], bt, vw[v]);
  }
}

// Vertices of degree in (kLowDeg, kMidDeg]: one warp per vertex.  Each lane
// keeps its (at most kMidPer) entries in registers; the labels are summed in
// the warp's open-addressing table in shared memory (at most kMidDeg + 1
// keys in kMidSlots slots), and only the slots used are reset afterwards.
// The rating is the one of k_cluster_high: the largest weight, then the
// smaller tie-hash, then the smaller label, own cluster included.
constexpr int kMidSlots = 512;
static_assert(kMidSlots >= 2 * (kMidDeg + 1), "mid-degree table at most half full");

// Adds weight w to label t's slot (claimed on first use); returns the slot,
// or -1 if the table were full (excluded by the bound above).
__device__ __forceinline__ int32_t mid_insert(int32_t* K, int32_t* V, int32_t t, int32_t w) {
  uint32_t h = slot_hash(t) & (uint32_t)(kMidSlots - 1);
  for (int probe = 0; probe < kMidSlots; probe++) {
    const int32_t prev = atomicCAS(&K[h], -1, t);
    if (prev == -1 || prev == t) {
      atomicAdd(&V[h], w);
      return (int32_t)h;
    }
    h = (h + 1) & (uint32_t)(kMidSlots - 1);
  }
  return -1;
}

__global__ void __launch_bounds__(kMidThreads) k_cluster_mid(GraphView g, const int32_t* __restrict__ hi, int32_t n_hi,
                                                             ClusterArgs a, uint32_t* err) {
  __shared__ int32_t sk[kMidWarps][kMidSlots];
  __shared__ int32_t sv[kMidWarps][kMidSlots];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* K = sk[warp];
  int32_t* V = sv[warp];
  for (int s = lane; s < kMidSlots; s += 32) {
    K[s] = -1;
    V[s] = 0;
  }
  __syncwarp();
  for (int64_t i = (int64_t)blockIdx.x * kMidWarps + warp; i < n_hi; i += (int64_t)gridDim.x * kMidWarps) {
    const int32_t v = hi[i];
    const int64_t beg = g.xadj[v];
    const int64_t deg = g.xadj[v + 1] - beg;
    if (deg > g.mid_deg) continue;
    if (!cluster_active(a, v, deg)) {
      if (lane == 0) a.req[v] = -1;
      continue;
    }
    const int32_t own = a.C[v];
    int32_t t[kMidPer], w[kMidPer], hs[kMidPer];
#pragma unroll
    for (int r = 0; r < kMidPer; r++) {
      const int j = lane + 32 * r;
      t[r] = j < deg ? g.adj[beg + j] : -1;
      w[r] = j < deg ? g.adjw[beg + j] : 0;
    }
#pragma unroll
    for (int r = 0; r < kMidPer; r++) t[r] = t[r] >= 0 ? a.C[t[r]] : -1;
    // the own cluster is a candidate even without an edge into it (weight 0)
    const int32_t ho = lane == 0 ? mid_insert(K, V, own, 0) : -1;
    bool lost = lane == 0 && ho < 0;
#pragma unroll
    for (int r = 0; r < kMidPer; r++) {
      hs[r] = t[r] >= 0 ? mid_insert(K, V, t[r], w[r]) : -1;
      lost |= t[r] >= 0 && hs[r] < 0;
    }
    if (lost) atomicOr(err, ERR_CAPACITY);
    __syncwarp();
    int32_t bs = ho >= 0 ? V[ho] : -1;
#pragma unroll
    for (int r = 0; r < kMidPer; r++)
      if (hs[r] >= 0) bs = max(bs, V[hs[r]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bs = max(bs, __shfl_xor_sync(0xffffffffu, bs, o));
    // among the labels with the best weight: the smallest (tie-hash, label)
    uint64_t bh = ~0ULL;
    int32_t bt = INT32_MAX;
    auto consider = [&](int32_t slot) {
      if (slot < 0 || V[slot] != bs) return;
      const int32_t x = K[slot];
      const uint64_t h = h_tie(a.seed, a.level, x);
      if (h < bh || (h == bh && x < bt)) {
        bh = h;
        bt = x;
      }
    };
    consider(ho);
#pragma unroll
    for (int r = 0; r < kMidPer; r++) consider(hs[r]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t oh = __shfl_xor_sync(0xffffffffu, bh, o);
      const int32_t ot = __shfl_xor_sync(0xffffffffu, bt, o);
      if (oh < bh || (oh == bh && ot < bt)) {
        bh = oh;
        bt = ot;
      }
    }
    __syncwarp();
    if (ho >= 0) {
      K[ho] = -1;
      V[ho] = 0;
    }
#pragma unroll
    for (int r = 0; r < kMidPer; r++)
      if (hs[r] >= 0) {
        K[hs[r]] = -1;
        V[hs[r]] = 0;
      }
    __syncwarp();
    if (lane == 0) cluster_request(a, v, own, bt, g.vw[v]);
  }
}

// 1: admitted without ordering (the whole demand fits), 2: contested.  The
// contested requests are also appended (in any order) as (target << 32 |
// tie-hash, id) pairs for the single-CTA resolution below.
__global__ void k_cluster_classify(int32_t n, const int32_t* __restrict__ req, const int32_t* __restrict__ Wc,
                                   const int32_t* __restrict__ ReqW, int64_t wcap, uint8_t* flag, uint64_t seed,
                                   int32_t level, uint64_t* key, int32_t* val, ClusterState* cs) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = req[v];
    uint8_t f = 0;
    if (t >= 0) f = ((int64_t)Wc[t] + ReqW[t] <= wcap) ? 1 : 2;
    flag[v] = f;
    if (f == 2) {
      const unsigned long long i = atomicAdd((unsigned long long*)&cs->ncont, 1ULL);
      const uint32_t hk = (uint32_t)(h_active(seed, level, (int32_t)v) >> 32);
      key[i] = ((uint64_t)(uint32_t)t << 32) | hk;
      val[i] = (int32_t)v;
    }
  }
}

// Contested requests, when there are at most kSmallThreads of them: one CTA
// orders them by (target, tie-hash, id) with a rank sort (the position of a
// request is the number of requests before it in that order, so the result
// does not depend on the append order) and admits each while the target's
// weight plus the requests up to it stay within the cap.  Longer lists take
// the multi-CTA path (scan compaction in id order, stable radix sort).
__global__ void __launch_bounds__(kSmallThreads) k_cluster_resolve(const uint64_t* __restrict__ key,
                                                                   const int32_t* __restrict__ val,
                                                                   const ClusterState* cs,
                                                                   const int32_t* __restrict__ Wc,
                                                                   const int32_t* __restrict__ vw, int64_t wcap,
                                                                   uint8_t* flag, cudaGraphConditionalHandle h_big) {
  __shared__ uint64_t sk[kSmallThreads];
  __shared__ int32_t sv[kSmallThreads];
  __shared__ uint64_t ok[kSmallThreads];
  __shared__ int32_t ov[kSmallThreads];
  __shared__ int64_t ex[kSmallThreads];
  __shared__ int64_t sm[33];
  const int64_t n64 = cs->ncont;
  if (threadIdx.x == 0) cudaGraphSetConditional(h_big, n64 > kSmallThreads ? 1u : 0u);
  if (n64 <= 0 || n64 > kSmallThreads) return;
  const int n = (int)n64, i = threadIdx.x;
  uint64_t ki = 0;
  int32_t vi = 0;
  if (i < n) {
    ki = key[i];
    vi = val[i];
    sk[i] = ki;
    sv[i] = vi;
  }
  __syncthreads();
  if (i < n) {
    int r = 0;
    for (int j = 0; j < n; j++) {
      const uint64_t kj = sk[j];
      r += (kj < ki || (kj == ki && sv[j] < vi)) ? 1 : 0;
    }
    ok[r] = ki;
    ov[r] = vi;
  }
  __syncthreads();
  const int64_t c = i < n ? (int64_t)vw[ov[i]] : 0;
  int64_t tot;
  const int64_t e = block_exclusive_scan(c, sm, &tot);
  ex[i] = e;
  __syncthreads();
  if (i < n) {
    const uint32_t t = (uint32_t)(ok[i] >> 32);
    int h = i;
    while (h > 0 && (uint32_t)(ok[h - 1] >> 32) == t) h--;  // first request of the same target
    flag[ov[i]] = ((int64_t)Wc[t] + (e + c - ex[h]) <= wcap) ? 1 : 0;
  }
}

struct LoadContested {
  const uint8_t* flag;
  __device__ int64_t operator()(int64_t i) const { return flag[i] == 2 ? 1 : 0; }
};
struct StoreContested {
  const int32_t* req;
  uint64_t seed;
  int32_t level;
  uint64_t* key;
  int32_t* val;
  __device__ void operator()(int64_t i, int64_t e, int64_t x) const {
    if (x) {
      const uint32_t hk = (uint32_t)(h_active(seed, level, (int32_t)i) >> 32);
      key[e] = ((uint64_t)(uint32_t)req[i] << 32) | hk;
      val[e] = (int32_t)i;
    }
  }
};
struct LoadSortedVw {
  const int32_t* val;
  const int32_t* vw;
  __device__ int64_t operator()(int64_t i) const { return vw[val[i]]; }
};

__global__ void k_cluster_heads(const uint64_t* __restrict__ key, const int64_t* __restrict__ P, const int64_t* d_n,
                                int64_t max_n, int64_t* headP) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n && i < max_n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t t = key[i] >> 32;
    if (i == 0 || (key[i - 1] >> 32) != t) headP[t] = P[i];
  }
}

__global__ void k_cluster_admit(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                                const int64_t* __restrict__ P, const int64_t* __restrict__ headP, const int64_t* d_n,
                                int64_t max_n, const int32_t* __restrict__ Wc, const int32_t* __restrict__ vw,
                                int64_t wcap, uint8_t* flag) {
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n && i < max_n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = (int32_t)(key[i] >> 32);
    const int32_t v = val[i];
    const int64_t inc = P[i] + vw[v] - headP[t];
    flag[v] = ((int64_t)Wc[t] + inc <= wcap) ? 1 : 0;
  }
}

__global__ void k_cluster_apply(int32_t n, const int32_t* __restrict__ req, const uint8_t* __restrict__ flag,
                                int32_t* C, int32_t* Wc, int32_t* ReqW, const int32_t* __restrict__ vw,
                                int64_t* moved, ClusterState* cs) {
  if (blockIdx.x == 0 && threadIdx.x == 0) cs->ncont = 0;  // for the next sub-round
  int32_t mine = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = req[v];
    if (t < 0) continue;
    ReqW[t] = 0;
    if (flag[v] != 1) continue;
    const int32_t cv = vw[v];
    atomicAdd(&Wc[C[v]], -cv);
    atomicAdd(&Wc[t], cv);
    C[v] = t;
    mine++;
  }
  mine = warp_sum(mine);  // one update of the shared counter per warp
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd((unsigned long long*)moved, (unsigned long long)mine);
}

// Iteration control of the clustering loop: stop after cluster_iters
// iterations or once fewer than 1 % of the vertices moved in one.
__global__ void k_cl_init(ClusterState* cs, int32_t iters, cudaGraphConditionalHandle h, int use_h) {
  cs->it = 0;
  cs->done = iters <= 0;
  cs->moved = 0;
  cs->kernels = 0;
  cs->ncont = 0;
  if (use_h) cudaGraphSetConditional(h, iters > 0 ? 1u : 0u);
}
__global__ void k_cl_begin(ClusterState* cs) { cs->moved = 0; }
__global__ void k_cl_end(ClusterState* cs, int32_t n, int32_t iters, cudaGraphConditionalHandle h, int use_h,
                         unsigned long long body_kernels) {
  cs->kernels += body_kernels;
  const bool stop = cs->moved * 100 < (int64_t)n || cs->it + 1 >= iters;
  cs->it += 1;
  cs->done = stop ? 1 : 0;
  if (use_h) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// isolated vertices: chunks of weight <= cap in id order, labelled n + chunk
struct LoadIsolated {
  const int64_t* xadj;
  const int32_t* vw;
  __device__ int64_t operator()(int64_t v) const { return xadj[v + 1] == xadj[v] ? vw[v] : 0; }
};
struct StoreIsolated {
  int32_t* C;
  const int32_t* vw;
  int32_t n;
  int64_t wcap;
  __device__ void operator()(int64_t v, int64_t s, int64_t x) const {
    if (!x) return;
    const int64_t first = s / wcap, last = (s + vw[v] - 1) / wcap;
    if (first == last) C[v] = (int32_t)(n + first);
  }
};

__global__ void k_mark_used(int32_t n, const int32_t* __restrict__ C, int32_t* used) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    used[C[v]] = 1;
}
struct LoadI32 {
  const int32_t* a;
  __device__ int64_t operator()(int64_t i) const { return a[i]; }
};
struct StoreRankI32 {
  int32_t* out;
  __device__ void operator()(int64_t i, int64_t e, int64_t) const { out[i] = (int32_t)e; }
};
__global__ void k_apply_rank(int32_t n, const int32_t* __restrict__ C, const int32_t* __restrict__ rank, int32_t* M) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    M[v] = rank[C[v]];
}

// ---------------------------------------------------------------------------
// contraction
// ---------------------------------------------------------------------------
__global__ void k_coarse_vw(int32_t n, const int32_t* __restrict__ M, const int32_t* __restrict__ vw, int32_t* vwc) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&vwc[M[v]], vw[v]);
}

// Keys (M(u), M(v)) and weights of the inter-cluster CSR entries, compacted
// to the front of the sort buffers.  Their order does not matter: parallel
// entries are summed after the sort.  A warp takes 32 consecutive vertices,
// whose rows form one contiguous range, and walks it 32 entries at a time;
// each lane finds the row of its entry among the 32 row starts.  A first walk
// counts the warp's valid entries, the block reserves one range for its eight
// warps with a single atomic, and a second walk (gathers now cached) writes.
// Rows of degree > mid_deg are jumped over (k_contract_keys_hub takes them),
// so that no warp walks a hub's row alone while the rest of its block waits.
__device__ __forceinline__ int contract_owner(int64_t x, int64_t b, int last) {
  // largest lane L <= last with row start(L) <= x (starts are non-decreasing)
  int lo = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int cand = lo + step;
    const int64_t s = __shfl_sync(0xffffffffu, b, cand > 31 ? 31 : cand);
    if (cand <= last && s <= x) lo = cand;
  }
  return lo;
}

// First entry at or after x0 that lies outside the rows of the lanes in
// `big` (E1 if none; warp-uniform, as x0 is).  The row holding x0 < E1 ends
// after x0, so every step advances.
__device__ __forceinline__ int64_t contract_skip(int64_t x0, int64_t E1, int64_t b, int64_t e, int last,
                                                 unsigned big) {
  while (big && x0 < E1) {
    const int o = contract_owner(x0, b, last);
    if (!((big >> o) & 1u)) break;
    x0 = __shfl_sync(0xffffffffu, e, o);
  }
  return x0;
}

__global__ void __launch_bounds__(kThreads) k_contract_keys(GraphView g, const int32_t* __restrict__ M, int bits,
                                                            uint64_t* key, int32_t* val, int64_t* valid) {
  constexpr int kWarps = kThreads / 32;
  __shared__ unsigned long long wcnt[kWarps];
  __shared__ unsigned long long bbase;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ntiles = ((int64_t)g.n + 31) / 32;
  for (int64_t bt = blockIdx.x; bt * kWarps < ntiles; bt += gridDim.x) {
    const int64_t tile = bt * kWarps + warp;
    int64_t E0 = 0, E1 = 0, b = 0, e = 0;
    int32_t mv = 0;
    int last = 0;
    unsigned big = 0;
    if (tile < ntiles) {  // warp-uniform
      const int64_t v = tile * 32 + lane;
      last = (int)min((int64_t)31, (int64_t)g.n - 1 - tile * 32);
      const bool vv = v < g.n;
      b = vv ? g.xadj[v] : 0;
      e = vv ? g.xadj[v + 1] : 0;
      mv = vv ? M[v] : 0;
      E0 = __shfl_sync(0xffffffffu, b, 0);
      E1 = __shfl_sync(0xffffffffu, e, last);
      big = __ballot_sync(0xffffffffu, e - b > g.mid_deg);
    }
    unsigned long long cnt = 0;
    for (int64_t x0 = contract_skip(E0, E1, b, e, last, big); x0 < E1;
         x0 = contract_skip(x0 + 32, E1, b, e, last, big)) {
      const int64_t x = x0 + lane;
      const int o = contract_owner(x, b, last);
      const int32_t mo = __shfl_sync(0xffffffffu, mv, o);
      const bool ok = x < E1 && !((big >> o) & 1u) && M[g.adj[x]] != mo;
      cnt += __popc(__ballot_sync(0xffffffffu, ok));
    }
    if (lane == 0) wcnt[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tot = 0;
      for (int w = 0; w < kWarps; w++) {
        const unsigned long long c = wcnt[w];
        wcnt[w] = tot;
        tot += c;
      }
      bbase = tot ? atomicAdd((unsigned long long*)valid, tot) : 0ULL;
    }
    __syncthreads();
    unsigned long long pos = bbase + wcnt[warp];
    for (int64_t x0 = contract_skip(E0, E1, b, e, last, big); x0 < E1;
         x0 = contract_skip(x0 + 32, E1, b, e, last, big)) {
      const int64_t x = x0 + lane;
      const int o = contract_owner(x, b, last);
      const int32_t mo = __shfl_sync(0xffffffffu, mv, o);
      const int32_t mu = (x < E1 && !((big >> o) & 1u)) ? M[g.adj[x]] : mo;
      const bool ok = mu != mo;
      const unsigned bal = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const unsigned long long p = pos + __popc(bal & lt);
        key[p] = ((uint64_t)(uint32_t)mo << bits) | (uint32_t)mu;
        val[p] = g.adjw[x];
      }
      pos += __popc(bal);
    }
    __syncthreads();  // wcnt and bbase are rewritten by the next round
  }
}

struct LoadHead {
  const uint64_t* key;
  const int64_t* d_valid;
  __device__ int64_t operator()(int64_t i) const {
    if (i >= *d_valid) return 0;
    return (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
  }
};
struct StoreHead {
  const uint64_t* key;
  uint64_t* ukey;
  int64_t* hstart;
  __device__ void operator()(int64_t i, int64_t e, int64_t x) const {
    if (x) {
      ukey[e] = key[i];
      hstart[e] = i;
    }
  }
};
struct LoadValid32 {
  const int32_t* val;
  const int64_t* d_valid;
  __device__ int64_t operator()(int64_t i) const { return i < *d_valid ? val[i] : 0; }
};

// Keys of the rows of degree > kMidDeg (one CTA per row; `sel` lists their
// positions in hi[]): the block counts its row's valid entries, reserves one
// range with a single atomic, and its warps fill it through a shared cursor.
// The rows of degree > mid_deg (flattened, in chunks of kHubChunk entries,
// kHubChunk / kThreads per thread): the rows of a chunk are looked up at once
// (one thread each), then every thread keys its entries, the block reserves
// one output range per chunk with a single atomic and each thread writes its
// valid entries at its exclusive prefix.
__global__ void __launch_bounds__(kThreads) k_contract_keys_hub(GraphView g, HubRows hr,
                                                                const int32_t* __restrict__ M, int bits,
                                                                uint64_t* key, int32_t* val, int64_t* valid) {
  constexpr int kPer = (int)(kHubChunk / kThreads);
  static_assert(kPer * kThreads == kHubChunk && kThreads >= kChunkRows, "chunk layout");
  __shared__ int64_t s_rb[kChunkRows], s_x0[kChunkRows];
  __shared__ int32_t s_mo[kChunkRows];
  __shared__ unsigned long long sm[33];
  __shared__ unsigned long long s_base;
  const int64_t m_hub = hr.pre[hr.n_huge];
  for (int64_t ch = blockIdx.x; ch < hr.nchunks; ch += gridDim.x) {
    const int64_t cb = ch * kHubChunk, ce = min(cb + kHubChunk, m_hub);
    const int32_t r = hr.chunk[ch] + (int32_t)threadIdx.x;
    bool row = false;
    if (threadIdx.x < kChunkRows && r < hr.n_huge) {
      const int64_t rb = hr.pre[r];
      row = rb < ce;
      if (row) {
        const int32_t u = hr.hi[hr.huge[r]];
        s_rb[threadIdx.x] = rb;
        s_x0[threadIdx.x] = g.xadj[u] - rb;  // CSR position of flat entry f: x0 + f
        s_mo[threadIdx.x] = M[u];
      }
    }
    const int nrows = __syncthreads_count(row);  // the chunk's rows are a prefix
    // entries f = cb + k * kThreads + threadIdx.x (coalesced), rows found by a
    // forward walk over the row starts
    int32_t mo[kPer], mu[kPer];
    int64_t xe[kPer];
    unsigned long long cnt = 0;
    int i = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      const int64_t f = cb + (int64_t)k * kThreads + threadIdx.x;
      mo[k] = 0;
      mu[k] = 0;
      xe[k] = -1;
      if (f < ce) {
        while (i + 1 < nrows && s_rb[i + 1] <= f) i++;
        xe[k] = s_x0[i] + f;
        mo[k] = s_mo[i];
        mu[k] = M[g.adj[xe[k]]];
        cnt += mu[k] != mo[k] ? 1 : 0;
      }
    }
    unsigned long long tot;
    unsigned long long pos = block_exclusive_scan(cnt, sm, &tot);
    if (threadIdx.x == 0) s_base = tot ? atomicAdd((unsigned long long*)valid, tot) : 0ULL;
    __syncthreads();
    pos += s_base;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      if (xe[k] < 0 || mu[k] == mo[k]) continue;
      key[pos] = ((uint64_t)(uint32_t)mo[k] << bits) | (uint32_t)mu[k];
      val[pos] = g.adjw[xe[k]];
      pos++;
    }
    __syncthreads();  // s_base and the row table are rewritten for the next chunk
  }
}

__global__ void k_copy_i64(const int64_t* src, int64_t* dst) { *dst = *src; }

__global__ void k_put_total(const int64_t* total, const int64_t* d_idx, int64_t* P) { P[*d_idx] = *total; }

__global__ void k_contract_fill(int64_t mc, const uint64_t* __restrict__ ukey, const int64_t* __restrict__ hstart,
                                const int64_t* __restrict__ P, const int64_t* d_valid, int bits, int32_t* adjc,
                                int32_t* adjwc) {
  const uint64_t mask = (1ULL << bits) - 1ULL;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < mc; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = hstart[u];
    const int64_t e = (u + 1 < mc) ? hstart[u + 1] : *d_valid;
    adjc[u] = (int32_t)(ukey[u] & mask);
    adjwc[u] = (int32_t)(P[e] - P[s]);
  }
}

__global__ void k_contract_xadj(int32_t nc, int64_t mc, const uint64_t* __restrict__ ukey, int bits, int64_t* xadjc) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= nc; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t target = (uint64_t)r << bits;
    int64_t lo = 0, hi = mc;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ukey[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    xadjc[r] = lo;
  }
}

__global__ void k_project(int32_t n, const int32_t* __restrict__ M, const int32_t* __restrict__ pic, int32_t* pi) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    pi[v] = pic[M[v]];
}

// ---------------------------------------------------------------------------
// initial mapping: breadth-first order in one CTA, cut into k weight chunks
// ---------------------------------------------------------------------------
constexpr int kInitSmemN = 12288;  // coarsest graphs up to this size keep the BFS state in shared memory

__global__ void __launch_bounds__(1024) k_initial(GraphView g, int32_t* order, int32_t* claim, int32_t* seen,
                                                  const int32_t* __restrict__ code_of_pe, int64_t k, int64_t cV,
                                                  int32_t* pi, uint32_t* err) {
  __shared__ int64_t sm[33];
  __shared__ int32_t s_tail, s_head, s_next;
  extern __shared__ __align__(16) int32_t init_smem[];
  const int32_t n = g.n;
  if (n <= kInitSmemN) {  // same algorithm, state on chip (the launch provides 3 * n words)
    order = init_smem;
    claim = init_smem + n;
    seen = init_smem + 2 * (size_t)n;
  }
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
    seen[v] = 0;
    claim[v] = INT32_MAX;
  }
  if (threadIdx.x == 0) {
    s_tail = 0;
    s_head = 0;
    s_next = 0;
  }
  __syncthreads();
  int64_t guard = 0;
  while (true) {
    const int32_t tail = s_tail;
    const int32_t head = s_head;
    if (tail >= n) break;
    if (++guard > 2 * (int64_t)n + 4) {  // cannot happen; bounded for safety
      if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
      break;
    }
    __syncthreads();
    if (head == tail) {  // next component: lowest unvisited id
      if (threadIdx.x == 0) {
        int32_t s = s_next;
        while (seen[s]) s++;
        s_next = s + 1;
        order[tail] = s;
        seen[s] = 1;
        s_tail = tail + 1;
      }
      __syncthreads();
      continue;
    }
    // one level: frontier [head, tail); children claimed by the earliest parent
    for (int32_t i = head + threadIdx.x; i < tail; i += blockDim.x) {
      const int32_t v = order[i];
      for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
        const int32_t u = g.adj[e];
        if (!seen[u]) atomicMin(&claim[u], i);
      }
    }
    __syncthreads();
    int64_t carry = 0;
    for (int32_t base = head; base < tail; base += blockDim.x) {
      const int32_t i = base + threadIdx.x;
      int64_t cnt = 0;
      if (i < tail) {
        const int32_t v = order[i];
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
          const int32_t u = g.adj[e];
          if (!seen[u] && claim[u] == i) cnt++;
        }
      }
      int64_t total;
      const int64_t ex = block_exclusive_scan(cnt, sm, &total);
      if (i < tail && cnt) {
        int64_t pos = tail + carry + ex;
        const int32_t v = order[i];
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; e++) {
          const int32_t u = g.adj[e];
          if (!seen[u] && claim[u] == i) order[pos++] = u;
        }
      }
      carry += total;
    }
    __syncthreads();
    for (int64_t j = tail + threadIdx.x; j < tail + carry; j += blockDim.x) {
      const int32_t u = order[j];
      seen[u] = 1;
      claim[u] = INT32_MAX;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_head = tail;
      s_tail = (int32_t)(tail + carry);
    }
    __syncthreads();
  }
  __syncthreads();
  // PE of the vertex whose preceding weight in breadth-first order is s
  int64_t carry = 0;
  for (int32_t base = 0; base < n; base += blockDim.x) {
    const int32_t i = base + threadIdx.x;
    const int64_t cv = (i < n) ? g.vw[order[i]] : 0;
    int64_t total;
    const int64_t ex = block_exclusive_scan(cv, sm, &total);
    if (i < n) pi[order[i]] = code_of_pe[((carry + ex) * k) / cV];
    carry += total;
  }
}

// high-degree hash-table sizes: next power of two >= 2 (deg + 1), at least 64
struct LoadTableSize {
  const int32_t* hi;
  const int64_t* xadj;
  __device__ int64_t operator()(int64_t i) const {
    const int32_t v = hi[i];
    const int64_t want = 2 * (xadj[v + 1] - xadj[v] + 1);
    int64_t s = 64;
    while (s < want) s <<= 1;
    return s;
  }
};

// read-backs go through the context's pinned block (slots 6 and 7 here):
// a pageable copy stages through a driver buffer that concurrent contexts share
int64_t read_i64(Ctx& c, const int64_t* d) {
  GM_CUDA(cudaMemcpyAsync(c.h_small + 6, d, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  return c.h_small[6];
}

int bits_for(int64_t x) {  // smallest b with x < 2^b
  int b = 0;
  while (b < 62 && (1LL << b) <= x) b++;
  return b;
}

void check_err(Ctx& c) {
  c.h_small[7] = 0;
  GM_CUDA(cudaMemcpyAsync(c.h_small + 7, c.errword, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  const uint32_t e = (uint32_t)(c.h_small[7] & 0xffffffffLL);
  if (e & ERR_TIMEOUT) throw ApiError(MAP_E_TIMEOUT, "a bounded device loop gave up");
  if (e) throw ApiError(MAP_E_INTERNAL, "device consistency check failed (flags " + std::to_string(e) + ")");
}

// One clustering sub-round: ratings and requests, classification, ordered
// admission of the contested requests, moves.
// adds the kernels of a conditional body that ran to the graph's count
__global__ void k_count_body(unsigned long long* kernels, unsigned long long n) { *kernels += n; }

void launch_subround(Ctx& c, int lvl, int32_t r, int64_t wcap) {
  Level& L = c.lv[lvl];
  const int32_t n = L.n;
  const unsigned gv = grid_for(c, kThreads, n);
  const unsigned gl = grid_for(c, kThreads / kSubWarp, n);
  uint8_t* flag = c.elig;
  int64_t* d_cont = c.counters + 6;
  const int kbits = bits_for(n) + 32;
  ClusterArgs a{c.C, c.Wc, c.ReqW, c.req, wcap, c.cfg.seed, c.cstate, lvl, r};
  c.prof_level = lvl;
  cudaEvent_t ev = c.prof_begin();
  k_cluster_tile<<<tile_grid(c, (const void*)k_cluster_tile, n), kTileThreads, 0, c.st>>>(view(L), a); count_launch();
  // per vertex: xadj 8, C 4, request 4 (+ hash, no memory); per entry: adjacency 4, weight 4, C(u) 4
  c.prof_end(ev, PK_CLUSTER, 16 * (int64_t)(L.n - L.n_hi) + 12 * (L.m - L.m_hi));
  // mid / high classes: xadj (8) of every listed vertex; the active half (the
  // sub-round's hash bit) also reads C and writes its request (8) and
  // streams its row (12 per entry): expected bytes
  if (L.n_hi > L.n_huge) {
    const int64_t nv = L.n_hi - L.n_huge, me = L.m_hi - L.m_huge;
    ev = c.prof_begin();
    k_cluster_mid<<<mid_grid(c, (const void*)k_cluster_mid, 0, L.n_hi), kMidThreads, 0, c.st>>>(view(L), L.hi,
                                                                                                L.n_hi, a, c.errword);
    count_launch();
    c.prof_end(ev, PK_CLUSTER_MID, 8 * nv + (8 * nv + 12 * me) / 2);
  }
  if (L.n_huge) {
    ev = c.prof_begin();
    const HubRows hr = hub_rows(L);
    // one wave of resident CTAs over the chunks
    const int64_t res = (int64_t)c.num_sms * c.resident_blocks((const void*)k_cluster_high, kHiThreads, 0);
    const unsigned gh = (unsigned)std::max<int64_t>(1, std::min<int64_t>(L.n_hub_chunks, res));
    k_cluster_high<<<gh, kHiThreads, 0, c.st>>>(view(L), hr, L.hi_off, c.htab, a, c.hub_ctr, c.errword);
    count_launch();
    const int64_t res2 = (int64_t)c.num_sms * c.resident_blocks((const void*)k_cluster_giant, kHiThreads, 0);
    k_cluster_giant<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(L.n_hub_chunks, res2)), kHiThreads, 0, c.st>>>(
        hr, L.hi_off, c.htab, L.hub_part, a, c.hub_ctr); count_launch();
    k_cluster_giant_finish<<<grid_for(c, kThreads, L.n_huge), kThreads, 0, c.st>>>(hr, L.hub_part, L.vw, a);
    count_launch();
    // the three launches of the class together
    c.prof_end(ev, PK_CLUSTER_HIGH, 8 * (int64_t)L.n_huge + (8 * (int64_t)L.n_huge + 12 * L.m_huge) / 2);
  }
  k_cluster_classify<<<gv, kThreads, 0, c.st>>>(n, c.req, c.Wc, c.ReqW, wcap, flag, c.cfg.seed, lvl, c.sort.key[0],
                                                c.sort.val[0], c.cstate); count_launch();
  // contested requests: compaction in id order, stable sort by (target,
  // tie-hash), per-target prefix, admission
  auto big = [&](cudaStream_t bs) {
    cudaStream_t saved = c.st;
    c.st = bs;
    scan(LoadContested{flag}, StoreContested{c.req, c.cfg.seed, lvl, c.sort.key[0], c.sort.val[0]}, n, nullptr,
         c.scan, bs);
    k_copy_i64<<<1, 1, 0, bs>>>(c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(n)), d_cont); count_launch();
    const int cur = radix_sort_pairs(c.sort, n, d_cont, kbits, bs, &c.cap, &c.cstate->kernels);
    scan(LoadSortedVw{c.sort.val[cur], L.vw}, StoreExcl{c.P64}, n, d_cont, c.scan, bs);
    k_cluster_heads<<<gv, kThreads, 0, bs>>>(c.sort.key[cur], c.P64, d_cont, n, c.headP); count_launch();
    k_cluster_admit<<<gv, kThreads, 0, bs>>>(c.sort.key[cur], c.sort.val[cur], c.P64, c.headP, d_cont, n, c.Wc,
                                             L.vw, wcap, flag); count_launch();
    c.st = saved;
  };
  if (c.cap.on()) {
    // a short list is resolved by one CTA; the multi-CTA path runs only for
    // longer ones (conditional node)
    cudaGraphConditionalHandle h = cap_handle(c.st, 0);
    k_cluster_resolve<<<1, kSmallThreads, 0, c.st>>>(c.sort.key[0], c.sort.val[0], c.cstate, c.Wc, L.vw, wcap, flag,
                                                     h); count_launch();
    long long body = 0;
    long long* outer = set_capture_counter(&body);
    cap_cond(c.cap, c.st, h, cudaGraphCondTypeIf, [&](cudaStream_t bs) {
      big(bs);
      k_count_body<<<1, 1, 0, bs>>>(&c.cstate->kernels, (unsigned long long)body + 1); count_launch();
    });
    set_capture_counter(outer);
  } else {
    big(c.st);  // stream launches: always the multi-CTA path (same admissions)
  }
  k_cluster_apply<<<gv, kThreads, 0, c.st>>>(n, c.req, flag, c.C, c.Wc, c.ReqW, L.vw, &c.cstate->moved,
                                             c.cstate); count_launch();
}

// Captures the clustering loop of one level: init; WHILE(continue) {
// sub-round 0; sub-round 1; stop test }.
void build_cluster_graph(Ctx& c, int lvl, int64_t wcap) {
  Level& L = c.lv[lvl];
  if (L.cgexec) cudaGraphExecDestroy(L.cgexec);
  L.cgexec = nullptr;
  const int32_t n = L.n;
  const unsigned gv = grid_for(c, kThreads, n);
  cudaStream_t saved = c.st;
  cap_streams(c);
  cudaStream_t cs = c.cap.s[0];
  long long root = 0, body = 0;
  long long* outer = set_capture_counter(&root);
  GM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  c.cap.depth = 0;
  c.st = cs;
  try {
    k_iota<<<gv, kThreads, 0, cs>>>(c.C, n); count_launch();
    GM_CUDA(cudaMemcpyAsync(c.Wc, L.vw, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, cs));
    GM_CUDA(cudaMemsetAsync(c.ReqW, 0, (size_t)n * sizeof(int32_t), cs));
    cudaGraphConditionalHandle h = cap_handle(cs, 0);
    k_cl_init<<<1, 1, 0, cs>>>(c.cstate, c.cfg.cluster_iters, h, 1); count_launch();
    cap_cond(c.cap, cs, h, cudaGraphCondTypeWhile, [&](cudaStream_t bs) {
      c.st = bs;
      set_capture_counter(&body);
      k_cl_begin<<<1, 1, 0, bs>>>(c.cstate); count_launch();
      launch_subround(c, lvl, 0, wcap);
      launch_subround(c, lvl, 1, wcap);
      k_cl_end<<<1, 1, 0, bs>>>(c.cstate, n, c.cfg.cluster_iters, h, 1, (unsigned long long)body + 1); count_launch();
      set_capture_counter(&root);
    });
    cudaGraph_t g = nullptr;
    GM_CUDA(cudaStreamEndCapture(cs, &g));
    c.cap.depth = -1;
    c.st = saved;
    set_capture_counter(outer);
    cudaError_t e = cudaGraphInstantiate(&L.cgexec, g, 0);
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
  L.cg_root = root;
}

// Clusters level `lvl`; returns n_c, fills L.M.
int32_t cluster_level(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  const int32_t n = L.n;
  const unsigned gv = grid_for(c, kThreads, n);
  const unsigned gl = grid_for(c, kThreads / kSubWarp, n);
  int64_t wcap = c.lmax / c.cfg.cluster_cap_div;
  if (wcap < L.max_vw) wcap = L.max_vw;
  if (wcap < 1) wcap = 1;
  // hash tables for the high-degree vertices
  if (L.n_hi) {
    if (!L.hi_off) L.hi_off = c.mem.make<int64_t>((size_t)L.n + 1);
    scan(LoadTableSize{L.hi, L.xadj}, StoreExcl{L.hi_off}, L.n_hi, nullptr, c.scan, c.st);
    const int64_t tiles = std::max<int64_t>(1, scan_tiles(L.n_hi));
    GM_CUDA(cudaMemcpyAsync(L.hi_off + L.n_hi, c.scan.tile_sums + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice,
                            c.st));
    L.hi_slots = read_i64(c, L.hi_off + L.n_hi);
    if (L.n_huge) {
      if (L.hi_slots > c.hcap) {
        if (c.htab) c.mem.put(c.htab);
        c.hcap = L.hi_slots;
        c.htab = c.mem.make<unsigned long long>((size_t)c.hcap);
        c.htab_clean = false;
      }
      // every sub-round leaves the tables empty; after a failure they are cleared again
      if (!c.htab_clean) GM_CUDA(cudaMemsetAsync(c.htab, 0xFF, (size_t)c.hcap * sizeof(unsigned long long), c.st));
      c.htab_clean = false;
    }
  }
  ClusterState* cs = c.cstate;
  bool graph_ran = false;
  if (c.use_graphs && !c.prof) {
    const int64_t key[8] = {(int64_t)L.n, L.m, (int64_t)L.n_hi | ((int64_t)L.n_huge << 32), L.hi_slots, wcap,
                            (int64_t)(intptr_t)c.htab, (int64_t)(intptr_t)L.hub_chunk, L.n_hub_chunks};
    bool same = L.cgexec != nullptr;
    for (int i = 0; i < 8 && same; i++) same = L.cg_key[i] == key[i];
    if (!same) {
      build_cluster_graph(c, lvl, wcap);
      for (int i = 0; i < 8; i++) L.cg_key[i] = key[i];
    }
    GM_CUDA(cudaGraphLaunch(L.cgexec, c.st));
    // read back with the cluster count below (kernel accounting only)
    GM_CUDA(cudaMemcpyAsync(c.h_cstate, cs, sizeof(ClusterState), cudaMemcpyDeviceToHost, c.st));
    graph_ran = true;
  } else {
    k_iota<<<gv, kThreads, 0, c.st>>>(c.C, n); count_launch();
    GM_CUDA(cudaMemcpyAsync(c.Wc, L.vw, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.st));
    GM_CUDA(cudaMemsetAsync(c.ReqW, 0, (size_t)n * sizeof(int32_t), c.st));
    k_cl_init<<<1, 1, 0, c.st>>>(cs, c.cfg.cluster_iters, 0, 0); count_launch();
    for (int32_t it = 0; it < c.cfg.cluster_iters; it++) {
      k_cl_begin<<<1, 1, 0, c.st>>>(cs); count_launch();
      launch_subround(c, lvl, 0, wcap);
      launch_subround(c, lvl, 1, wcap);
      k_cl_end<<<1, 1, 0, c.st>>>(cs, n, c.cfg.cluster_iters, 0, 0, 0); count_launch();
      GM_CUDA(cudaMemcpyAsync(c.h_cstate, cs, sizeof(ClusterState), cudaMemcpyDeviceToHost, c.st));
      GM_CUDA(cudaStreamSynchronize(c.st));
      if (c.h_cstate->done) break;
    }
  }
  // isolated vertices, then number the clusters by ascending label
  scan(LoadIsolated{L.xadj, L.vw}, StoreIsolated{c.C, L.vw, n, wcap}, n, nullptr, c.scan, c.st);
  const int64_t nlab = 2 * (int64_t)n + 1;
  GM_CUDA(cudaMemsetAsync(c.rank, 0, (size_t)nlab * sizeof(int32_t), c.st));
  k_mark_used<<<gv, kThreads, 0, c.st>>>(n, c.C, c.rank); count_launch();
  scan(LoadI32{c.rank}, StoreRankI32{c.rank}, nlab, nullptr, c.scan, c.st);
  // the cluster count and the error flags with one synchronisation
  GM_CUDA(cudaMemcpyAsync(c.h_small, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(nlab)), sizeof(int64_t),
                          cudaMemcpyDeviceToHost, c.st));
  c.h_small[1] = 0;
  GM_CUDA(cudaMemcpyAsync(c.h_small + 1, c.errword, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.st));
  if (!L.M) L.M = c.mem.make<int32_t>((size_t)std::max(1, n));
  k_apply_rank<<<gv, kThreads, 0, c.st>>>(n, c.C, c.rank, L.M); count_launch();
  GM_CUDA(cudaGetLastError());
  GM_CUDA(cudaStreamSynchronize(c.st));
  if (graph_ran) add_launches(L.cg_root + (long long)c.h_cstate->kernels);
  const int64_t nc = c.h_small[0];
  const uint32_t e = (uint32_t)(c.h_small[1] & 0xffffffffLL);
  if (e & ERR_TIMEOUT) throw ApiError(MAP_E_TIMEOUT, "a bounded device loop gave up");
  if (e) throw ApiError(MAP_E_INTERNAL, "device consistency check failed (flags " + std::to_string(e) + ")");
  c.htab_clean = true;
  return (int32_t)nc;
}

// Builds level lvl + 1 from level lvl and its M.
void free_level(Ctx& c, Level& L) {
  drop_graph(L);
  if (L.cgexec) cudaGraphExecDestroy(L.cgexec);
  L.cgexec = nullptr;
  for (void* p : {(void*)L.xadj, (void*)L.adj, (void*)L.adjw, (void*)L.vw, (void*)L.pi, (void*)L.hi,
                  (void*)L.huge, (void*)L.hi_off, (void*)L.M, (void*)L.hub_pre, (void*)L.hub_chunk,
                  (void*)L.hub_part, (void*)L.hub_sidx, (void*)L.hub_split, (void*)L.hub_gtab,
                  (void*)L.hub_acc})
    if (p) c.mem.put(p);
  L = Level{};
}

// Builds level lvl + 1 from level lvl and its M.  `spare` is the level that
// held this index before (repeated runs): its buffers are reused when the
// sizes match, which also keeps its instantiated refinement graph valid.
void contract_level(Ctx& c, int lvl, int32_t nc, Level* spare) {
  Level& F = c.lv[lvl];
  Level C;
  const bool reuse_n = spare && spare->n == nc;
  if (reuse_n) {
    C = *spare;
    *spare = Level{};
  } else if (spare) {
    free_level(c, *spare);
  }
  C.n = nc;
  const int64_t m = F.m;
  const unsigned gv = grid_for(c, kThreads, F.n);
  if (!reuse_n) C.vw = c.mem.make<int32_t>((size_t)std::max(1, nc));
  GM_CUDA(cudaMemsetAsync(C.vw, 0, (size_t)std::max(1, nc) * sizeof(int32_t), c.st));
  k_coarse_vw<<<gv, kThreads, 0, c.st>>>(F.n, F.M, F.vw, C.vw); count_launch();
  const int bits = bits_for(nc);  // ids < 2^bits - 1, so the all-ones key is free
  int64_t* d_valid = c.counters + 7;
  GM_CUDA(cudaMemsetAsync(d_valid, 0, sizeof(int64_t), c.st));
  int64_t mc = 0;
  if (!reuse_n) C.xadj = c.mem.make<int64_t>((size_t)nc + 1);
  const int64_t old_m = reuse_n ? C.m : -1;
  if (m > 0) {
    k_contract_keys<<<grid_for(c, kThreads, F.n), kThreads, 0, c.st>>>(view(F), F.M, bits, c.sort.key[0],
                                                                       c.sort.val[0], d_valid); count_launch();
    if (F.n_huge) {
      k_contract_keys_hub<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(F.n_hub_chunks, (int64_t)c.num_sms * 8)),
                            kThreads, 0, c.st>>>(view(F), hub_rows(F), F.M, bits, c.sort.key[0], c.sort.val[0],
                                                 d_valid); count_launch();
    }
    c.prof_level = lvl;
    cudaEvent_t ev = c.prof_begin();
    const int cur = radix_sort_pairs(c.sort, m, d_valid, 2 * bits, c.st);  // the valid keys only
    // per 8-bit pass: keys read twice (histogram, scatter), key + value read and written once
    c.prof_end(ev, PK_SORT, (int64_t)((2 * bits + 7) / 8) * m * (8 + 12 + 12));
    uint64_t* skey = c.sort.key[cur];
    int32_t* sval = c.sort.val[cur];
    uint64_t* ukey = c.sort.key[cur ^ 1];
    scan(LoadHead{skey, d_valid}, StoreHead{skey, ukey, c.P64b}, m, nullptr, c.scan, c.st);
    mc = read_i64(c, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(m)));
    scan(LoadValid32{sval, d_valid}, StoreExcl{c.P64}, m, nullptr, c.scan, c.st);
    // P64[valid] = total weight of the valid entries
    k_put_total<<<1, 1, 0, c.st>>>(c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(m)), d_valid, c.P64); count_launch();
    if (old_m != mc) {
      if (C.adj) c.mem.put(C.adj);
      if (C.adjw) c.mem.put(C.adjw);
      drop_graph(C);
      C.adj = c.mem.make<int32_t>((size_t)std::max<int64_t>(1, mc));
      C.adjw = c.mem.make<int32_t>((size_t)std::max<int64_t>(1, mc));
    }
    if (mc > 0)
      k_contract_fill<<<grid_for(c, kThreads, mc), kThreads, 0, c.st>>>(mc, ukey, c.P64b, c.P64, d_valid, bits, C.adj,
                                                                       C.adjw); count_launch();
    k_contract_xadj<<<grid_for(c, kThreads, nc + 1), kThreads, 0, c.st>>>(nc, mc, ukey, bits, C.xadj); count_launch();
  } else {
    if (!C.adj) C.adj = c.mem.make<int32_t>(1);
    if (!C.adjw) C.adjw = c.mem.make<int32_t>(1);
    if (old_m != 0) drop_graph(C);
    GM_CUDA(cudaMemsetAsync(C.xadj, 0, ((size_t)nc + 1) * sizeof(int64_t), c.st));
  }
  C.m = mc;
  if (!reuse_n) C.pi = c.mem.make<int32_t>((size_t)std::max(1, nc));
  GM_CUDA(cudaMemsetAsync(C.pi, 0, (size_t)std::max(1, nc) * sizeof(int32_t), c.st));
  GM_CUDA(cudaGetLastError());
  c.lv.push_back(C);
}

__global__ void k_max_i32(int32_t n, const int32_t* __restrict__ a, int32_t* out) {
  int32_t m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = a[i] > m ? a[i] : m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int32_t y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}



}  // namespace

void coarsen_alloc(Ctx& c) {
  const size_t n = (size_t)std::max(1, c.n0);
  c.cstate = c.mem.make<ClusterState>(1);
  static_assert(sizeof(ClusterState) <= kPinnedBlock, "pinned block too small");
  if (!c.h_cstate) c.h_cstate = static_cast<ClusterState*>(pinned_get(sizeof(ClusterState)));
  c.C = c.mem.make<int32_t>(n);
  c.Wc = c.mem.make<int32_t>(n);
  c.ReqW = c.mem.make<int32_t>(n);
  c.req = c.mem.make<int32_t>(n);
  c.rank = c.mem.make<int32_t>(2 * n + 2);
  c.hub_ctr = c.mem.make<unsigned long long>(2);
  GM_CUDA(cudaMemsetAsync(c.hub_ctr, 0, 2 * sizeof(unsigned long long), c.st));
}

void validate_graph(Ctx& c) {
  Level& L = c.lv[0];
  unsigned long long* sums = reinterpret_cast<unsigned long long*>(c.counters);
  GM_CUDA(cudaMemsetAsync(c.errword, 0, sizeof(uint32_t), c.st));
  GM_CUDA(cudaMemsetAsync(sums, 0, 4 * sizeof(int64_t), c.st));  // weights; searching / other entries
  k_validate_rows<<<grid_for(c, kThreads, L.n), kThreads, 0, c.st>>>(view(L), L.m, c.errword, sums); count_launch();
  // the entries only once the rows are known to be sound (their search needs a monotone xadj)
  int64_t* hs = c.h_small;
  hs[0] = 0;
  GM_CUDA(cudaMemcpyAsync(hs, c.errword, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  if (hs[0] == 0 && L.m > 0) {
    k_validate_entries<<<grid_for(c, kThreads, (L.m + kValChunk - 1) / kValChunk), kThreads, 0, c.st>>>(
        view(L), L.m, c.errword, sums); count_launch();
  }
  // the largest vertex weight in the same round trip
  int32_t* dmax = reinterpret_cast<int32_t*>(c.counters + 4);
  GM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int64_t), c.st));
  k_max_i32<<<grid_for(c, kThreads, L.n), kThreads, 0, c.st>>>(L.n, L.vw, dmax); count_launch();
  GM_CUDA(cudaGetLastError());
  // pinned: [0] error flags, [1..2] sums, [3] largest weight, [4..5] searching / other entries
  hs[0] = 0;
  hs[3] = 0;
  GM_CUDA(cudaMemcpyAsync(hs, c.errword, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(hs + 1, sums, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(hs + 3, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(hs + 4, sums + 2, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  uint32_t e = (uint32_t)(hs[0] & 0xffffffffLL);
  if (hs[4] != hs[5]) e |= ERR_ASYM;  // an entry without its twin
  const unsigned long long h[2] = {(unsigned long long)hs[1], (unsigned long long)hs[2]};
  const int32_t hmax = (int32_t)(hs[3] & 0xffffffffLL);
  GM_CUDA(cudaMemsetAsync(sums, 0, 4 * sizeof(int64_t), c.st));
  if (e) {
    std::string m = "invalid graph:";
    if (e & ERR_XADJ) m += " xadj not monotone or out of range;";
    if (e & ERR_RANGE) m += " adjacency index out of range;";
    if (e & ERR_SELFLOOP) m += " self-loop;";
    if (e & ERR_UNSORTED) m += " row not strictly ascending (duplicate edge?);";
    if (e & ERR_ASYM) m += " missing or differently weighted reverse edge;";
    if (e & ERR_WEIGHT) m += " weight < 1;";
    throw ApiError(MAP_E_INVALID, m);
  }
  if (h[0] >= (1ULL << 31) || h[1] >= (1ULL << 31))
    throw ApiError(MAP_E_OVERFLOW, "sum of vertex weights and sum of edge weights must be < 2^31");
  c.cV = (int64_t)h[0];
  L.max_vw = hmax;
}

int32_t coarsen(Ctx& c) {
  c.level_gen++;
  // previous coarse levels are kept as spares: repeated runs on the same
  // graph rebuild identical levels into the same buffers
  std::vector<Level> spare(c.lv.begin() + 1, c.lv.end());
  c.lv.resize(1);
  while ((int32_t)c.lv.size() < c.cfg.max_levels &&
         (int64_t)c.lv.back().n >= (int64_t)c.cfg.coarsest_factor * c.k) {
    const int lvl = (int)c.lv.size() - 1;
    const int32_t nc = c.cfg.coarsener == 1 ? match_level(c, lvl) : cluster_level(c, lvl);
    Level& F = c.lv[lvl];
    if ((int64_t)nc * c.cfg.stall_den > (int64_t)c.cfg.stall_num * F.n) {
      c.mem.put(F.M);
      F.M = nullptr;
      break;
    }
    contract_level(c, lvl, nc, lvl < (int)spare.size() ? &spare[lvl] : nullptr);
    classify_degrees(c, (int)c.lv.size() - 1);  // also the level's largest vertex weight
  }
  for (Level& L : spare) free_level(c, L);
  return (int32_t)c.lv.size();
}

void initial_map(Ctx& c) {
  Level& L = c.lv.back();
  if (c.cfg.initial == 1) {  // hierarchical multisection of the coarsest graph
    hm_run(c, (int)c.lv.size() - 1, 8, &c.hm_init);
    return;
  }
  if (L.n > kInitSmemN && initial_map_large(c)) return;
  const size_t smem = L.n <= kInitSmemN ? (size_t)3 * L.n * sizeof(int32_t) : 0;
  static std::atomic<unsigned long long> attr_done{0};  // one bit per device
  const unsigned long long bit = 1ULL << (c.dev & 63);
  if (!(attr_done.load() & bit)) {
    GM_CUDA(cudaFuncSetAttribute(k_initial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(3 * kInitSmemN * sizeof(int32_t))));
    attr_done.fetch_or(bit);
  }
  k_initial<<<1, 1024, smem, c.st>>>(view(L), c.C, c.req, c.Wc, c.d_code_of_pe, c.k, c.cV, L.pi, c.errword); count_launch();
  GM_CUDA(cudaGetLastError());
  check_err(c);
}

void project(Ctx& c, int lvl) {
  Level& F = c.lv[lvl];
  const Level& C = c.lv[lvl + 1];
  k_project<<<grid_for(c, kThreads, F.n), kThreads, 0, c.st>>>(F.n, F.M, C.pi, F.pi); count_launch();
  GM_CUDA(cudaGetLastError());
}

}  // namespace gm
