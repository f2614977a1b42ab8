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

}  // namespace gm
