// Non-template parts of the device primitives (see prim.cuh).
#include <atomic>

#include "prim.cuh"

namespace gm {


static std::atomic<long long> g_launches{0};
static thread_local long long* t_capture_counter = nullptr;
// While a graph is being captured, launches are counted into the capture's
// counter instead: they run later, as graph nodes, and are added then.
void count_launch() {
  if (t_capture_counter) ++*t_capture_counter;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long* set_capture_counter(long long* p) {
  long long* old = t_capture_counter;
  t_capture_counter = p;
  return old;
}

__global__ void __launch_bounds__(1024) k_scan_tile_sums(int64_t* tile_sums, int64_t ntiles) {
  __shared__ int64_t sm[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = (i < ntiles) ? tile_sums[i] : 0;
    int64_t total;
    int64_t e = block_exclusive_scan(v, sm, &total);
    if (i < ntiles) tile_sums[i] = carry + e;
    carry += total;
  }
  if (threadIdx.x == 0) tile_sums[ntiles] = carry;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint64_t* __restrict__ keys, int64_t max_n,
                                                            const int64_t* d_n, int shift,
                                                            int64_t* __restrict__ hist, int64_t max_tiles,
                                                            int64_t skip_upto) {
  __shared__ int32_t cnt[256];
  int64_t n = load_count(d_n, max_n);
  if (n <= skip_upto) n = 0;  // the single-CTA sort handles it
  for (int i = threadIdx.x; i < 256; i += kSortThreads) cnt[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base < n) {
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
      int64_t idx = base + i;
      if (idx < n) atomicAdd(&cnt[(int)((keys[idx] >> shift) & 255u)], 1);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kSortThreads) hist[(int64_t)d * max_tiles + blockIdx.x] = cnt[d];
}

// Stable scatter: within a tile, items are ordered (warp, item, lane), which is
// the global index order; ranks among equal digits follow that order.  The
// tile is first placed in digit order in shared memory, then written out so
// that consecutive threads write consecutive positions of a digit's run
// (coalesced stores instead of one scattered store per item).
constexpr size_t kScatterSmem = (size_t)kSortTile * (sizeof(uint64_t) + sizeof(int32_t));
static_assert(kSortThreads == 256, "one digit per thread in the tile's digit scan");
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint64_t* __restrict__ kin,
                                                               const int32_t* __restrict__ vin,
                                                               uint64_t* __restrict__ kout,
                                                               int32_t* __restrict__ vout, int64_t max_n,
                                                               const int64_t* d_n, int shift,
                                                               const int64_t* __restrict__ hist_off,
                                                               int64_t max_tiles, int64_t skip_upto) {
  extern __shared__ __align__(16) unsigned char scatter_raw[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(scatter_raw);      // [kSortTile]
  int32_t* sv = reinterpret_cast<int32_t*>(sk + kSortTile);      // [kSortTile]
  __shared__ int32_t wcnt[kSortWarps][256];
  __shared__ int64_t goff[256];
  __shared__ int32_t tstart[256];
  __shared__ int32_t sm32[33];
  const int64_t n = load_count(d_n, max_n);
  if (n <= skip_upto) return;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= n) return;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  for (int d = threadIdx.x; d < 256; d += kSortThreads) goff[d] = hist_off[(int64_t)d * max_tiles + blockIdx.x];
  __syncthreads();

  uint64_t k[kSortItems];
  int32_t v[kSortItems];
  int32_t rank[kSortItems];
  const unsigned lt = (1u << l) - 1u;
  const int64_t wbase = base + (int64_t)w * 32 * kSortItems;
#pragma unroll
  for (int j = 0; j < kSortItems; j++) {
    int64_t idx = wbase + j * 32 + l;
    bool valid = idx < n;
    k[j] = valid ? kin[idx] : 0;
    v[j] = valid ? vin[idx] : 0;
    int d = valid ? (int)((k[j] >> shift) & 255u) : 256 + l;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int r = 0;
    if (valid) r = wcnt[w][d] + __popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0) wcnt[w][d] += __popc(peers);
    __syncwarp();
    rank[j] = valid ? r : -1;
  }
  __syncthreads();
  // per digit: the warps' offsets within the digit, and the digit's count
  int32_t dcount = 0;
  for (int d = threadIdx.x; d < 256; d += kSortThreads) {
    int32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kSortWarps; ww++) {
      int32_t t = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += t;
    }
    dcount = run;
  }
  // digit starts within the tile (kSortThreads == 256: one digit per thread)
  int32_t total;
  const int32_t ex = block_exclusive_scan(dcount, sm32, &total);
  tstart[threadIdx.x] = ex;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortItems; j++) {
    if (rank[j] >= 0) {
      const int d = (int)((k[j] >> shift) & 255u);
      const int p = tstart[d] + wcnt[w][d] + rank[j];
      sk[p] = k[j];
      sv[p] = v[j];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < total; i += kSortThreads) {
    const uint64_t key = sk[i];
    const int d = (int)((key >> shift) & 255u);
    const int64_t pos = goff[d] + (i - tstart[d]);
    kout[pos] = key;
    vout[pos] = sv[i];
  }
}

// Single CTA: stable LSD radix sort of n <= kSmallSort pairs in shared memory.
// Items of warp w are [w * items, (w + 1) * items) in lane-strided order, so
// (warp, item, lane) order is index order and equal digits keep it.
__global__ void __launch_bounds__(kSmallThreads) k_sort_small(const uint64_t* __restrict__ kin,
                                                              const int32_t* __restrict__ vin,
                                                              uint64_t* __restrict__ kout,
                                                              int32_t* __restrict__ vout, const int64_t* d_n,
                                                              int64_t max_n, int bits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* ks = reinterpret_cast<uint64_t*>(smem_raw);                  // [2][kSmallSort]
  int32_t* vs = reinterpret_cast<int32_t*>(ks + 2 * kSmallSort);          // [2][kSmallSort]
  int32_t* wcnt = vs + 2 * kSmallSort;                                    // [kW][256]
  __shared__ int32_t dbase[257];
  __shared__ int64_t sm[33];
  const int64_t n64 = load_count(d_n, max_n);
  if (n64 > kSmallSort || n64 <= 0) return;
  const int n = (int)n64;
  for (int i = threadIdx.x; i < n; i += kSmallThreads) {
    ks[i] = kin[i];
    vs[i] = vin[i];
  }
  const int cur = cta_sort_small(ks, vs, wcnt, dbase, sm, n, bits);
  for (int i = threadIdx.x; i < n; i += kSmallThreads) {
    kout[i] = ks[cur * kSmallSort + i];
    vout[i] = vs[cur * kSmallSort + i];
  }
}

void sort_init() {
  static std::atomic<unsigned long long> done{0};  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ULL << (dev & 63);
  if (done.load() & bit) return;
  cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small_sort_smem());
  cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
  done.fetch_or(bit);
}

cudaGraphConditionalHandle cap_handle(cudaStream_t st, unsigned int default_value) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(st, &status, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
      status != cudaStreamCaptureStatusActive)
    throw std::runtime_error("cap_handle: stream is not capturing");
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, default_value, cudaGraphCondAssignDefault) != cudaSuccess)
    throw std::runtime_error("cap_handle: cudaGraphConditionalHandleCreate failed");
  return h;
}

__global__ void k_sort_gate(const int64_t* d_n, cudaGraphConditionalHandle h, unsigned long long* kcount,
                            unsigned long long body_kernels) {
  const bool big = *d_n > kSmallSort;
  cudaGraphSetConditional(h, big ? 1u : 0u);
  if (big && kcount) atomicAdd(kcount, body_kernels);
}

static void sort_passes(SortBufs& b, int64_t max_n, const int64_t* d_n, int bits, int64_t skip, cudaStream_t st) {
  const int64_t tiles = sort_tiles(max_n);
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    k_sort_hist<<<(unsigned)tiles, kSortThreads, 0, st>>>(b.key[cur], max_n, d_n, shift, b.hist, tiles, skip); count_launch();
    scan(LoadI64{b.hist}, StoreExcl{b.hist_off}, 256 * tiles, nullptr, b.scan, st);
    k_sort_scatter<<<(unsigned)tiles, kSortThreads, kScatterSmem, st>>>(b.key[cur], b.val[cur], b.key[cur ^ 1],
                                                             b.val[cur ^ 1], max_n, d_n, shift, b.hist_off,
                                                             tiles, skip); count_launch();
    cur ^= 1;
  }
}

int radix_sort_pairs(SortBufs& b, int64_t max_n, const int64_t* d_n, int bits, cudaStream_t st, Capture* cap,
                     unsigned long long* kcount) {
  if (max_n <= 0 || bits <= 0) return 0;
  const int passes = (bits + 7) / 8;
  const int out = passes & 1;  // buffer holding the result after `passes` swaps
  sort_init();
  if (!d_n) {
    if (max_n <= kSmallSort) {
      k_sort_small<<<1, kSmallThreads, small_sort_smem(), st>>>(b.key[0], b.val[0], b.key[out], b.val[out], nullptr,
                                                                max_n, bits); count_launch();
    } else {
      sort_passes(b, max_n, nullptr, bits, -1, st);
    }
    return out;
  }
  // device-counted: the single-CTA kernel takes counts <= kSmallSort and
  // writes into the result buffer; the multi-CTA passes skip those counts
  k_sort_small<<<1, kSmallThreads, small_sort_smem(), st>>>(b.key[0], b.val[0], b.key[out], b.val[out], d_n, max_n,
                                                            bits); count_launch();
  if (max_n <= kSmallSort) return out;
  if (cap && cap->on()) {
    cudaGraphConditionalHandle h = cap_handle(st, 0);
    k_sort_gate<<<1, 1, 0, st>>>(d_n, h, kcount, (unsigned long long)passes * 5); count_launch();
    long long body = 0;
    long long* outer = set_capture_counter(&body);
    cap_cond(*cap, st, h, cudaGraphCondTypeIf,
             [&](cudaStream_t bs) { sort_passes(b, max_n, d_n, bits, kSmallSort, bs); });
    set_capture_counter(outer);
    if (body != (long long)passes * 5) throw std::runtime_error("radix_sort_pairs: unexpected pass kernel count");
  } else {
    sort_passes(b, max_n, d_n, bits, kSmallSort, st);
  }
  return out;
}

}  // namespace gm
