// Deterministic device primitives: block reductions, a three-phase exclusive
// scan over int64 values produced by a functor, and a stable LSD radix sort of
// (uint64 key, int32 value) pairs.  Element counts may live in device memory
// (``d_n``) so that data-dependent sizes need no host round trip; grids are
// sized for the host-known upper bound ``max_n`` and tiles past the count
// exit at once.  These are the building blocks of the contraction (sort +
// segmented reduce), cluster admission and rebalancing selection.
#pragma once

#include <stdexcept>

#include "common.cuh"

namespace gm {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

__device__ __forceinline__ int64_t load_count(const int64_t* d_n, int64_t max_n) {
  return d_n ? *d_n : max_n;
}

// ---------------------------------------------------------------------------
// block-wide helpers (blockDim.x multiple of 32, <= 1024)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T>
__device__ T block_sum(T v, T* sm /* >= 32 */) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  T r = 0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? sm[l] : T(0);
    r = warp_sum(r);
    if (l == 0) sm[0] = r;
  }
  __syncthreads();
  r = sm[0];
  __syncthreads();
  return r;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total.
template <class T>
__device__ T block_exclusive_scan(T v, T* sm /* >= 33 */, T* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    T s = (l < nw) ? sm[l] : T(0);
    T t = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += y;
    }
    if (l < nw) sm[l] = t - s;
    if (l == 31) sm[32] = t;
  }
  __syncthreads();
  T r = sm[w] + x - v;
  *total = sm[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// scan: out(i, exclusive prefix, value) for i < n, plus total
// ---------------------------------------------------------------------------
template <class Load>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Load load, int64_t max_n, const int64_t* d_n,
                                                              int64_t* tile_sums) {
  __shared__ int64_t sm[33];
  const int64_t n = load_count(d_n, max_n);
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  if (base < n) {
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
      int64_t idx = base + i;
      if (idx < n) s += load(idx);
    }
  }
  s = block_sum(s, sm);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = (base < n) ? s : 0;
}

// single block: exclusive scan of tile sums in place, total to tile_sums[ntiles]
__global__ void __launch_bounds__(1024) k_scan_tile_sums(int64_t* tile_sums, int64_t ntiles);

template <class Load, class Store>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(Load load, Store store, int64_t max_n,
                                                             const int64_t* d_n, const int64_t* tile_off) {
  __shared__ int64_t sm[33];
  const int64_t n = load_count(d_n, max_n);
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (base >= n) return;
  int64_t vals[kScanItems];
  int64_t local = 0;
  const int64_t first = base + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    int64_t idx = first + j;
    vals[j] = (idx < n) ? load(idx) : 0;
    local += vals[j];
  }
  int64_t total;
  int64_t run = block_exclusive_scan(local, sm, &total) + tile_off[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    int64_t idx = first + j;
    if (idx < n) store(idx, run, vals[j]);
    run += vals[j];
  }
}

struct ScanTmp {
  int64_t* tile_sums = nullptr;  // >= tiles(max_n) + 1
};

__host__ inline int64_t scan_tiles(int64_t max_n) { return (max_n + kScanTile - 1) / kScanTile; }

// Exclusive scan; the total lands in tmp.tile_sums[tiles] (device).
template <class Load, class Store>
void scan(Load load, Store store, int64_t max_n, const int64_t* d_n, ScanTmp tmp, cudaStream_t st) {
  int64_t tiles = scan_tiles(max_n);
  if (tiles == 0) tiles = 1;
  k_scan_reduce<<<(unsigned)tiles, kScanThreads, 0, st>>>(load, max_n, d_n, tmp.tile_sums); count_launch();
  k_scan_tile_sums<<<1, 1024, 0, st>>>(tmp.tile_sums, tiles); count_launch();
  k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, st>>>(load, store, max_n, d_n, tmp.tile_sums); count_launch();
}

// common functors
struct LoadI64 {
  const int64_t* a;
  __device__ int64_t operator()(int64_t i) const { return a[i]; }
};
struct StoreExcl {
  int64_t* out;
  __device__ void operator()(int64_t i, int64_t e, int64_t) const { out[i] = e; }
};

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
struct SortBufs {
  uint64_t* key[2] = {nullptr, nullptr};
  int32_t* val[2] = {nullptr, nullptr};
  int64_t* hist = nullptr;      // 256 * max_tiles
  int64_t* hist_off = nullptr;  // 256 * max_tiles
  ScanTmp scan;                 // for 256 * max_tiles elements
  int64_t capacity = 0;         // elements
};

__host__ inline int64_t sort_tiles(int64_t max_n) { return (max_n + kSortTile - 1) / kSortTile; }

// Single-CTA sort of device-counted sets of at most kSmallSort elements
// (stable LSD radix sort in shared memory); larger sets take the multi-CTA
// passes, whose kernels return at once when the count is small.
constexpr int kSmallSort = 4096;
constexpr int kSmallThreads = 1024;
__host__ inline size_t small_sort_smem() {
  return (size_t)2 * kSmallSort * (sizeof(uint64_t) + sizeof(int32_t)) +
         (size_t)(kSmallThreads / 32) * 256 * sizeof(int32_t);
}

__global__ void k_sort_hist(const uint64_t* __restrict__ keys, int64_t max_n, const int64_t* d_n, int shift,
                            int64_t* __restrict__ hist, int64_t max_tiles, int64_t skip_upto);
__global__ void k_sort_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                               uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t max_n,
                               const int64_t* d_n, int shift, const int64_t* __restrict__ hist_off,
                               int64_t max_tiles, int64_t skip_upto);
// Stable LSD radix sort of n <= kSmallSort (key, value) pairs held in the
// double buffers ks[2][kSmallSort], vs[2][kSmallSort] of shared memory, by
// key bits [0, bits), by one CTA of kSmallThreads threads.  wcnt holds
// (kSmallThreads / 32) * 256 counters, dbase 257, sm 33.  Returns the buffer
// index holding the result.  Items of warp w are [w * items, (w + 1) * items)
// in lane-strided order, so (warp, item, lane) order is index order and equal
// digits keep it.
// Up to kRankSortMax pairs are ordered by a rank sort instead (the position of
// pair i is the number of pairs with a smaller key, or an equal key and a
// smaller index: the same stable order at a cost that grows with n instead of
// the radix passes' fixed cost over kSmallSort slots).
constexpr int kRankSortMax = 512;
__device__ __forceinline__ int cta_sort_small(uint64_t* ks, int32_t* vs, int32_t* wcnt, int32_t* dbase, int64_t* sm,
                                              int n, int bits) {
  constexpr int kW = kSmallThreads / 32;
  constexpr int kItems = kSmallSort / kSmallThreads;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const unsigned lt = (1u << l) - 1u;
  if (n <= kRankSortMax) {
    const uint64_t mask = bits >= 64 ? ~0ULL : ((1ULL << bits) - 1ULL);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kSmallThreads) {
      const uint64_t ki = ks[i] & mask;
      int r = 0;
      for (int j = 0; j < n; j++) {
        const uint64_t kj = ks[j] & mask;
        r += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
      }
      ks[kSmallSort + r] = ks[i];
      vs[kSmallSort + r] = vs[i];
    }
    __syncthreads();
    return 1;
  }
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    const uint64_t* kc = ks + cur * kSmallSort;
    const int32_t* vc = vs + cur * kSmallSort;
    uint64_t* kn = ks + (cur ^ 1) * kSmallSort;
    int32_t* vn = vs + (cur ^ 1) * kSmallSort;
    for (int i = threadIdx.x; i < kW * 256; i += kSmallThreads) wcnt[i] = 0;
    __syncthreads();
    int rank[kItems], dig[kItems];
#pragma unroll
    for (int j = 0; j < kItems; j++) {
      const int idx = w * 32 * kItems + j * 32 + l;
      const bool valid = idx < n;
      const int d = valid ? (int)((kc[idx] >> shift) & 255u) : 256 + l;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      int r = 0;
      if (valid) r = wcnt[w * 256 + d] + __popc(peers & lt);
      __syncwarp();
      if (valid && (peers & lt) == 0) wcnt[w * 256 + d] += __popc(peers);
      __syncwarp();
      rank[j] = valid ? r : -1;
      dig[j] = d;
    }
    __syncthreads();
    int64_t tot = 0;
    if (threadIdx.x < 256) {
      int32_t run = 0;
      for (int ww = 0; ww < kW; ww++) {
        const int32_t t = wcnt[ww * 256 + threadIdx.x];
        wcnt[ww * 256 + threadIdx.x] = run;
        run += t;
      }
      tot = run;
    }
    int64_t all;
    const int64_t ex = block_exclusive_scan(tot, sm, &all);
    if (threadIdx.x < 256) dbase[threadIdx.x] = (int32_t)ex;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kItems; j++) {
      if (rank[j] < 0) continue;
      const int idx = w * 32 * kItems + j * 32 + l;
      const int pos = dbase[dig[j]] + wcnt[w * 256 + dig[j]] + rank[j];
      kn[pos] = kc[idx];
      vn[pos] = vc[idx];
    }
    __syncthreads();
    cur ^= 1;
  }
  return cur;
}

__global__ void k_sort_small(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, int32_t* __restrict__ vout, const int64_t* d_n,
                             int64_t max_n, int bits);
void sort_init();

// ---------------------------------------------------------------------------
// stream capture into graphs with conditional nodes
// ---------------------------------------------------------------------------
// s[d] captures at nesting depth d (0: the root graph); depth < 0: no capture.
struct Capture {
  cudaStream_t s[6] = {};
  int depth = -1;
  bool on() const { return depth >= 0; }
};

// A conditional handle on the graph currently captured by `st`.
cudaGraphConditionalHandle cap_handle(cudaStream_t st, unsigned int default_value);

// Appends a conditional node (IF / WHILE on handle h) to the graph captured by
// `st` and captures `body(stream)` into its body graph.
template <class F>
void cap_cond(Capture& cap, cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
              F&& body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(st, &status, nullptr, &g, &deps, &ed, &nd) != cudaSuccess ||
      status != cudaStreamCaptureStatusActive)
    throw std::runtime_error("cap_cond: stream is not capturing");
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, ed, nd, &p) != cudaSuccess)
    throw std::runtime_error("cap_cond: cudaGraphAddNode failed");
  if (cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    throw std::runtime_error("cap_cond: cudaStreamUpdateCaptureDependencies failed");
  cudaGraph_t bg = p.conditional.phGraph_out[0];
  const int d = ++cap.depth;
  cudaStream_t bs = cap.s[d];
  if (cudaStreamBeginCaptureToGraph(bs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    throw std::runtime_error("cap_cond: cudaStreamBeginCaptureToGraph failed");
  body(bs);
  if (cudaStreamEndCapture(bs, &bg) != cudaSuccess) throw std::runtime_error("cap_cond: cudaStreamEndCapture failed");
  --cap.depth;
}

// Sorts buffer 0 (n elements, count on device or max_n) by key bits [0, bits).
// Returns the buffer index (0 or 1) that holds the sorted result.  While
// `cap` is capturing, the multi-CTA passes sit in a conditional node that
// runs only for device counts above kSmallSort.
// kcount (device, may be NULL) accumulates the kernels run by the
// conditional passes, so that graph executions can be counted.
int radix_sort_pairs(SortBufs& b, int64_t max_n, const int64_t* d_n, int bits, cudaStream_t st,
                     Capture* cap = nullptr, unsigned long long* kcount = nullptr);

}  // namespace gm
