// Degree classes of the per-vertex kernels.
//
// A vertex of degree <= kLowDeg is handled inside a warp tile (tile.cuh).  A
// vertex with kLowDeg < degree <= kMidDeg gets one warp (kMidWarps vertices
// per block at a time, no block-wide barrier per vertex); each lane keeps its
// at most kMidPer CSR entries in registers.  Vertices of larger degree keep a
// whole CTA.
#pragma once

#include "common.cuh"

namespace gm {

constexpr int kMidDeg = 255;
constexpr int kMidPer = (kMidDeg + 31) / 32;
constexpr int kMidWarps = 8;
constexpr int kMidThreads = kMidWarps * 32;
// bound (in 32-bit words) of one warp's dense connectivity table (PE codes and
// level group sums): kMidWarps tables stay within 48 KB of shared memory
constexpr int kMidTableMax = 1536;
// entries per chunk when the rows of degree > kMidDeg are spread over CTAs
constexpr int64_t kHubChunk = 2048;
// chunks a CTA takes at once in the connectivity-table and exact-change
// kernels: the rows of such a span are checked in one step, one thread each
// (a row's check is a chain of dependent loads; per chunk it set the pace)
constexpr int64_t kSpanChunks = 4;
constexpr int kSpanRows = 256;  // rows of one span at most (rows there have more than kLowDeg + 1 entries)
static_assert(kSpanChunks * kHubChunk / 34 + 2 <= kSpanRows, "a span's rows fit the per-span row table");
// rows rated by one CTA whole (PE-code tables); larger rows sum chunk tables
constexpr int64_t kSplitDeg = 4096;
// bound of the per-level partial tables of the larger rows (else rated whole)
constexpr int64_t kSplitTableBytes = 1LL << 30;

// Dynamic chunk tickets: thread 0 draws the next chunk for the CTA.  The
// last CTA to leave resets the counters for the next launch (every CTA's
// final draw precedes its exit count).
__device__ __forceinline__ int64_t next_chunk(unsigned long long* ctr, int64_t* s_ch) {
  if (threadIdx.x == 0) *s_ch = (int64_t)atomicAdd(&ctr[0], 1ULL);
  __syncthreads();
  const int64_t ch = *s_ch;
  __syncthreads();
  return ch;
}
__device__ __forceinline__ void leave_chunks(unsigned long long* ctr) {
  if (threadIdx.x == 0 && atomicAdd(&ctr[1], 1ULL) == gridDim.x - 1) {
    ctr[0] = 0;
    ctr[1] = 0;
  }
}

}  // namespace gm
