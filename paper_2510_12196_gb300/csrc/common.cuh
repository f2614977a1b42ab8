// Shared device definitions of the GB300 mapping library (sm_103a).
//
// PE code space.  The hierarchy a_1:...:a_l (Section 2) is re-encoded so that
// every level owns a fixed bit field: PE p with digits x_i = floor(p /
// (a_1...a_{i-1})) mod a_i gets the code sum_i x_i << shift_i, shift_i =
// sum_{j<i} ceil(log2 a_j).  The code is strictly increasing in p (so "lowest
// PE id" tie-breaks become "lowest code"), the level-i group of a code is
// code >> s_i with s_i = shift_i + bits_i, and the distance of two different
// PEs (d_i for the smallest level whose group holds both) depends only on the
// highest differing bit:  D(x, y) = dist_of_bit[31 - clz(x ^ y)], D(x, x) = 0.
// All device state stores mappings as codes; ids are converted at the ABI.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cg = cooperative_groups;

namespace gm {

constexpr int kMaxLevels = 16;     // hierarchy depth limit
constexpr int kMaxCodeBits = 14;   // code space <= 16384 PEs (dense shared-memory tables)
constexpr int kSubWarp = 8;        // lanes per low-degree vertex
constexpr int kSlots = 4;          // edges per lane held in registers
constexpr int kLowDeg = kSubWarp * kSlots;  // degree handled by the sub-warp path
constexpr int kBuckets = 64;       // rebalancing loss buckets (0:+, 1:0, 2+floor(log2(-g)))
constexpr int kBucketBits = 6;

struct Topo {
  int32_t levels;
  int32_t k;           // number of PEs
  int32_t code_bits;   // total bits
  int32_t kc;          // 1 << code_bits
  int32_t s[kMaxLevels + 1];           // s[i] = cumulative bits through level i (s[0] = 0)
  int32_t dist_of_bit[32];
  int32_t dist[kMaxLevels];
};

// Distance in code space (see file comment).
__device__ __forceinline__ int32_t dcode(const int32_t* __restrict__ sdist, int32_t x, int32_t y) {
  uint32_t z = (uint32_t)(x ^ y);
  return z ? sdist[31 - __clz(z)] : 0;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) output for state seed ^ x.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t seed, uint64_t x) {
  uint64_t z = (seed ^ x) + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// Hash streams: salt in bits 60..63, level above bit 32 (above bit 52 for the
// rebalancing stream, whose iteration counter sits in bits 32..51).
__host__ __device__ __forceinline__ uint64_t h_active(uint64_t seed, int32_t level, int32_t v) {
  return mix64(seed, (1ULL << 60) | ((uint64_t)level << 32) | (uint64_t)(uint32_t)v);
}
__host__ __device__ __forceinline__ uint64_t h_tie(uint64_t seed, int32_t level, int32_t t) {
  return mix64(seed, (2ULL << 60) | ((uint64_t)level << 32) | (uint64_t)(uint32_t)t);
}
__host__ __device__ __forceinline__ uint64_t h_rebalance(uint64_t seed, int32_t level, int32_t t, int32_t v) {
  return mix64(seed, (3ULL << 60) | ((uint64_t)level << 52) | ((uint64_t)(t & 0xFFFFF) << 32) |
                         (uint64_t)(uint32_t)v);
}

// Loss bucket of the rebalancing gain g (log2-spaced, Section 4.2).
__device__ __forceinline__ int32_t loss_bucket(int64_t g) {
  if (g > 0) return 0;
  if (g == 0) return 1;
  return 2 + (63 - __clzll((unsigned long long)(-g)));
}

// Load the topology's distance-by-bit table into shared memory.
__device__ __forceinline__ void load_sdist(int32_t* sdist, const Topo& t) {
  for (int i = threadIdx.x; i < 32; i += blockDim.x) sdist[i] = t.dist_of_bit[i];
}

// Error word written by device-side checks (bit flags, host maps them to a status).
enum : uint32_t {
  ERR_RANGE = 1u,       // adjacency out of range
  ERR_SELFLOOP = 2u,
  ERR_UNSORTED = 4u,    // row not strictly ascending (duplicates)
  ERR_ASYM = 8u,        // missing or differently weighted reverse edge
  ERR_WEIGHT = 16u,     // weight < 1
  ERR_XADJ = 32u,       // xadj not monotone
  ERR_CAPACITY = 64u,   // internal table overflow
  ERR_TIMEOUT = 128u,   // a bounded device wait gave up
};

// Process-wide count of kernels launched by this library (host side).  Graph
// executions are added after they complete (add_launches); while a graph is
// captured, count_launch counts into the capture counter that is set.
void count_launch();
long long launch_count();
void add_launches(long long n);
long long* set_capture_counter(long long* p);

// Small pinned host blocks (kPinnedBlock bytes) shared by all contexts.
// cudaFreeHost synchronises the whole device, so a context returns its
// blocks to a process-wide free list instead of freeing them.
constexpr size_t kPinnedBlock = 4096;
void* pinned_get(size_t bytes);
void pinned_put(void* p);

}  // namespace gm

#define GM_CUDA(x)                                                          \
  do {                                                                      \
    cudaError_t _e = (x);                                                   \
    if (_e != cudaSuccess) throw gm::CudaError(_e, #x, __FILE__, __LINE__); \
  } while (0)
