// Allocation-free evaluation of the objective J and the maximum block weight.
//
// map_objective_noalloc computes the same two numbers as map_objective, but
// without a context and without allocating any device memory: the caller
// passes device pointers to the graph, the mapping and a two-element output,
// and the scratch (J accumulator, block weights, PE code table) lives in one
// file-scope __device__ array.  It serves callers that cannot or must not
// allocate: the CUDA allocation calls (cudaMalloc / cudaFree) may synchronise
// the whole device and stall unrelated streams, and some callers run under a
// fixed device-memory budget owned by their own memory pool, or simply hold a
// graph and a mapping in device memory and want its cost without creating a
// context (whose set-up allocates and validates the whole graph).
//
// Limits and sharing: at most kNoAllocMaxPE = 16384 PEs (code space 2^14).
// Every call on a device shares the single scratch array, which keeps the
// last call's contents; each call clears what must start at zero before it
// uses it.  Calls whose work overlaps on the GPU (different streams, or
// several host threads) race on the array and give wrong results: serialise
// them.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and keeps it for the
// process; make that first call before any stream capture on the device.
// A cudaDeviceReset invalidates the kept address: the entry point must not be
// used on a device after it was reset.
#include <mutex>
#include <string>

#include "engine.h"

namespace gm {
namespace {

constexpr int kNoAllocMaxPE = 1 << kMaxCodeBits;
constexpr int kNaThreads = 256;

struct NoAllocScratch {
  unsigned long long J;
  long long maxw;
  long long W[kNoAllocMaxPE];       // block weights by PE code
  int32_t code[kNoAllocMaxPE];      // PE id -> PE code
};

// The scratch of every call on this device (about 192 KiB, held until exit).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

struct Hier {
  int32_t a[kMaxLevels];
};

// Clears the accumulators and fills the PE id -> code table.
__global__ void k_na_clear(NoAllocScratch* s, Topo t, Hier h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    s->J = 0;
    s->maxw = 0;
  }
  for (int b = i; b < t.kc; b += gridDim.x * blockDim.x) s->W[b] = 0;
  for (int p = i; p < t.k; p += gridDim.x * blockDim.x) {
    int rem = p, code = 0;
    for (int l = 0; l < t.levels; l++) {
      code |= (rem % h.a[l]) << t.s[l];
      rem /= h.a[l];
    }
    s->code[p] = code;
  }
}

// J and block weights: one 8-lane sub-warp per vertex (any degree); mapping
// entries or neighbours outside their range are skipped, and every row is
// clamped to [0, xadj[n]) so that a malformed xadj cannot read outside the
// adjacency arrays.
__global__ void __launch_bounds__(kNaThreads) k_na_eval(int32_t n, const int64_t* __restrict__ xadj,
                                                        const int32_t* __restrict__ adj,
                                                        const int32_t* __restrict__ adjw,
                                                        const int32_t* __restrict__ vw,
                                                        const int32_t* __restrict__ pi, NoAllocScratch* s, Topo t) {
  __shared__ int32_t sdist[32];
  __shared__ int64_t sm[33];
  load_sdist(sdist, t);
  __syncthreads();
  auto tile = cg::tiled_partition<kSubWarp>(cg::this_thread_block());
  const int lane = tile.thread_rank();
  const int64_t nsw = ((int64_t)gridDim.x * blockDim.x) / kSubWarp;
  int64_t acc = 0;
  const int64_t m = xadj[n];
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kSubWarp; v < n; v += nsw) {
    const int32_t pv = pi[v];
    if (pv < 0 || pv >= t.k) continue;
    const int32_t cv = s->code[pv];
    if (lane == 0) atomicAdd((unsigned long long*)&s->W[cv], (unsigned long long)(int64_t)vw[v]);
    const int64_t eb = max(xadj[v], (int64_t)0), ee = min(xadj[v + 1], m);
    for (int64_t e = eb + lane; e < ee; e += kSubWarp) {
      const int32_t u = adj[e];
      if (u < 0 || u >= n) continue;
      const int32_t pu = pi[u];
      if (pu < 0 || pu >= t.k) continue;
      acc += (int64_t)(adjw ? adjw[e] : 1) * dcode(sdist, cv, s->code[pu]);
    }
  }
  acc = block_sum(acc, sm);
  if (threadIdx.x == 0 && acc) atomicAdd(&s->J, (unsigned long long)acc);
}

__global__ void k_na_finish(NoAllocScratch* s, int32_t kc, int64_t* out) {
  __shared__ long long smax[32];
  long long mx = 0;
  for (int b = threadIdx.x; b < kc; b += blockDim.x) mx = s->W[b] > mx ? s->W[b] : mx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = smax[w] > mx ? smax[w] : mx;
    s->maxw = mx;
    out[0] = (int64_t)s->J;
    out[1] = mx;
  }
}

// Address of the scratch array on each device, looked up once per device.
std::mutex g_na_mutex;
NoAllocScratch* g_na_ptr[256] = {nullptr};

}  // namespace
}  // namespace gm

using namespace gm;

extern "C" GPUMAP_API map_status map_objective_noalloc(const int64_t* xadj, const int32_t* adjncy,
                                                       const int32_t* adjwgt, const int32_t* vwgt, int32_t n,
                                                       const int32_t* pi, const int32_t* hier, const int32_t* dist,
                                                       int32_t levels, int64_t* out, void* stream) {
  last_create_error().clear();
  auto fail = [](map_status s, const std::string& m) {
    last_create_error() = m;  // readable through map_last_error(NULL)
    return s;
  };
  if (n < 1 || !xadj || !vwgt || !pi || !hier || !dist || !out) return fail(MAP_E_INVALID, "null pointer or n < 1");
  if (levels < 1 || levels > kMaxLevels) return fail(MAP_E_INVALID, "levels must be in [1, 16]");
  Topo t{};
  Hier h{};
  t.levels = levels;
  int64_t k = 1;
  int32_t s = 0;
  for (int i = 0; i < levels; i++) {
    if (hier[i] < 1 || dist[i] < 0) return fail(MAP_E_INVALID, "hierarchy factors must be >= 1, distances >= 0");
    int32_t b = 0;
    while ((1 << b) < hier[i]) b++;
    t.s[i] = s;
    s += b;
    if (s > kMaxCodeBits)
      return fail(MAP_E_INVALID, "hierarchy exceeds the 16384-PE code space of map_objective_noalloc");
    k *= hier[i];
    h.a[i] = hier[i];
    t.dist[i] = dist[i];
  }
  t.s[levels] = s;
  t.code_bits = s;
  t.kc = 1 << s;
  t.k = (int32_t)k;
  for (int b = 0; b < 32; b++) t.dist_of_bit[b] = 0;
  for (int i = 0; i < levels; i++)
    for (int b = t.s[i]; b < t.s[i + 1]; b++) t.dist_of_bit[b] = dist[i];

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return fail(MAP_E_CUDA, "cudaGetDevice failed");
  }
  NoAllocScratch* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(MAP_E_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                    cudaGetErrorString(e));
      }
      g_na_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  k_na_clear<<<(t.kc + kNaThreads - 1) / kNaThreads, kNaThreads, 0, st>>>(scratch, t, h); count_launch();
  int64_t blocks = ((int64_t)n + kNaThreads / kSubWarp - 1) / (kNaThreads / kSubWarp);
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  k_na_eval<<<(unsigned)blocks, kNaThreads, 0, st>>>(n, xadj, adjncy, adjwgt, vwgt, pi, scratch, t); count_launch();
  k_na_finish<<<1, 256, 0, st>>>(scratch, t.kc, out); count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MAP_E_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  return MAP_OK;
}
