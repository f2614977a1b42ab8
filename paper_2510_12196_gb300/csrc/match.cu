// Coarsening by two-hop matching (Section 4.2, "Matching"): heavy-edge
// rounds with the exp*2 rating w(u,v)^2 / (c(u) c(v)), then, while at most
// 75% of the vertices are matched, leaf, twin and relative stages and the
// pairing of isolated vertices.
//
// Heavy-edge round: one 8-lane sub-warp per unmatched vertex scans its
// unmatched neighbours u with c(v) + c(u) <= L_max for the largest rating,
// compared exactly as w1^2 c(u2) against w2^2 c(u1) in 128-bit integers
// (c(v) cancels); equal ratings go to the smaller edge hash (the
// deterministic noise), then the smaller u.  v and u are matched when each
// prefers the other.  Rounds repeat until one matches nothing.
//
// Two-hop stage: the still unmatched vertices of the stage append (group, id)
// keys (leaf: the neighbour; twin: the top 31 bits of the neighbour-set hash;
// relative: the neighbour of smallest (degree, id); isolated: 0); a stable
// radix sort orders them, and consecutive members of a group pair up (1st
// with 2nd, 3rd with 4th, ...) when their weights fit L_max and, for twins,
// their neighbour sets are equal.  Every decision is a function of values,
// so the result equals a serial evaluation.
#include <algorithm>
#include <string>

#include "engine.h"

namespace gm {
namespace {

constexpr int kMThreads = 256;

struct MatchGraph {
  int32_t n;
  const int64_t* __restrict__ xadj;
  const int32_t* __restrict__ adj;
  const int32_t* __restrict__ adjw;
  const int32_t* __restrict__ vw;
};

__device__ __forceinline__ uint64_t h_edge(uint64_t seed, int32_t level, int32_t a, int32_t b) {
  return mix64(seed ^ ((4ULL << 60) | ((uint64_t)(uint32_t)level << 48)),
               ((uint64_t)(uint32_t)a << 32) | (uint32_t)b);
}
__device__ __forceinline__ uint64_t h_nbr(uint64_t seed, int32_t u) {
  return mix64(seed, (5ULL << 60) | (uint64_t)(uint32_t)u);
}

// candidate (w, c, u) of vertex v better than (bw, bc, bu)?
__device__ __forceinline__ bool rate_better(int64_t w, int64_t c, int32_t u, int64_t bw, int64_t bc, int32_t bu,
                                            int32_t v, uint64_t seed, int32_t level) {
  if (u < 0) return false;
  if (bu < 0) return true;
  const unsigned __int128 lhs = (unsigned __int128)(uint64_t)(w * w) * (uint64_t)bc;
  const unsigned __int128 rhs = (unsigned __int128)(uint64_t)(bw * bw) * (uint64_t)c;
  if (lhs != rhs) return lhs > rhs;
  const uint64_t hu = h_edge(seed, level, min(v, u), max(v, u));
  const uint64_t hb = h_edge(seed, level, min(v, bu), max(v, bu));
  return hu < hb || (hu == hb && u < bu);
}

__global__ void __launch_bounds__(kMThreads) k_match_prefer(MatchGraph g, const int32_t* __restrict__ mate,
                                                             int64_t lmax, uint64_t seed, int32_t level,
                                                             int32_t* __restrict__ pref) {
  const int sl = threadIdx.x & (kSubWarp - 1);
  const int64_t nsw = ((int64_t)gridDim.x * blockDim.x) / kSubWarp;
  // the whole warp iterates together (the shuffles below take every lane)
  const int64_t first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kSubWarp;
  const int64_t wfirst = first - (first % (32 / kSubWarp));
  for (int64_t w0 = wfirst; w0 < g.n; w0 += nsw) {
    const int64_t v0 = w0 + (first - wfirst);
    const bool free_v = v0 < g.n && mate[v0] < 0;
    const int32_t v = (int32_t)v0;
    int64_t bw = 0, bc = 0;
    int32_t bu = -1;
    if (free_v) {
      const int64_t cv = g.vw[v];
      for (int64_t x = g.xadj[v] + sl; x < g.xadj[v + 1]; x += kSubWarp) {
        const int32_t u = g.adj[x];
        if (mate[u] >= 0) continue;
        const int64_t cu = g.vw[u];
        if (cv + cu > lmax) continue;
        const int64_t w = g.adjw[x];
        if (rate_better(w, cu, u, bw, bc, bu, v, seed, level)) {
          bw = w;
          bc = cu;
          bu = u;
        }
      }
    }
#pragma unroll
    for (int o = kSubWarp / 2; o > 0; o >>= 1) {
      const int64_t ow = __shfl_xor_sync(0xffffffffu, bw, o);
      const int64_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
      const int32_t ou = __shfl_xor_sync(0xffffffffu, bu, o);
      if (rate_better(ow, oc, ou, bw, bc, bu, v, seed, level)) {
        bw = ow;
        bc = oc;
        bu = ou;
      }
    }
    if (sl == 0 && v0 < g.n) pref[v] = free_v ? bu : -1;
  }
}

// warp-aggregated addition to a device counter
__device__ __forceinline__ void count_add(int64_t* ctr, int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0 && x) atomicAdd((unsigned long long*)ctr, (unsigned long long)x);
}

__global__ void k_match_mutual(int32_t n, const int32_t* __restrict__ pref, int32_t* mate, int64_t* ctr) {
  int64_t mine = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = pref[v];
    if (u >= 0 && pref[u] == (int32_t)v) {
      mate[v] = u;
      mine++;
    }
  }
  count_add(ctr, mine);
}

// keys ((group << idbits) | v) of the unmatched vertices of a two-hop stage,
// appended in any order (the sort orders them)
__global__ void k_twohop_keys(MatchGraph g, const int32_t* __restrict__ mate, int stage, uint64_t seed, int idbits,
                              uint64_t* key, int32_t* val, int64_t* cnt) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < g.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    bool take = false;
    uint64_t grp = 0;
    if (v < g.n && mate[v] < 0) {
      const int64_t b = g.xadj[v], e = g.xadj[v + 1], d = e - b;
      if (stage == 1) {  // leaves
        take = d == 1;
        if (take) grp = (uint32_t)g.adj[b];
      } else if (stage == 2) {  // twins
        take = d >= 2;
        if (take) {
          uint64_t h = 0;
          for (int64_t x = b; x < e; x++) h += h_nbr(seed, g.adj[x]);
          grp = h >> 33;
        }
      } else if (stage == 3) {  // relatives: the matchmaker
        take = d >= 1;
        if (take) {
          int32_t mm = -1;
          int64_t md = 0;
          for (int64_t x = b; x < e; x++) {
            const int32_t u = g.adj[x];
            const int64_t du = g.xadj[u + 1] - g.xadj[u];
            if (mm < 0 || du < md || (du == md && u < mm)) {
              mm = u;
              md = du;
            }
          }
          grp = (uint32_t)mm;
        }
      } else {  // isolated
        take = d == 0;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    unsigned long long pos = 0;
    if (lane == 0 && bal) pos = atomicAdd((unsigned long long*)cnt, (unsigned long long)__popc(bal));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (take) {
      const unsigned long long p = pos + __popc(bal & lt);
      key[p] = (grp << idbits) | (uint64_t)v;
      val[p] = (int32_t)v;
    }
  }
}

__device__ __forceinline__ bool same_neighbours(const MatchGraph& g, int32_t a, int32_t b) {
  const int64_t da = g.xadj[a + 1] - g.xadj[a];
  if (da != g.xadj[b + 1] - g.xadj[b]) return false;
  for (int64_t i = 0; i < da; i++)
    if (g.adj[g.xadj[a] + i] != g.adj[g.xadj[b] + i]) return false;
  return true;
}

// consecutive members of each group of the sorted keys pair up
__global__ void k_pair_groups(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                              const int64_t* __restrict__ cnt, int idbits, MatchGraph g, int64_t lmax, int twins,
                              int32_t* mate, int64_t* matched) {
  const int64_t c = *cnt;
  int64_t mine = 0;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < c; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    if (i < c) {
      const uint64_t grp = key[i] >> idbits;
      // first member of the group: lower bound of (grp << idbits)
      int64_t lo = 0, hi = i;
      const uint64_t first = grp << idbits;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key[mid] < first) lo = mid + 1;
        else hi = mid;
      }
      if (((i - lo) & 1) == 0 && i + 1 < c && (key[i + 1] >> idbits) == grp) {
        const int32_t a = val[i], b = val[i + 1];
        if ((int64_t)g.vw[a] + g.vw[b] <= lmax && (!twins || same_neighbours(g, a, b))) {
          mate[a] = b;
          mate[b] = a;
          mine += 2;
        }
      }
    }
    count_add(matched, mine);
    mine = 0;
  }
}

struct LoadRep {
  const int32_t* mate;
  __device__ int64_t operator()(int64_t v) const {
    const int32_t m = mate[v];
    return (m < 0 || (int64_t)m > v) ? 1 : 0;  // v represents its pair (or itself)
  }
};
struct StoreRank {
  int32_t* rank;
  __device__ void operator()(int64_t v, int64_t e, int64_t x) const {
    if (x) rank[v] = (int32_t)e;
  }
};
__global__ void k_match_number(int32_t n, const int32_t* __restrict__ mate, const int32_t* __restrict__ rank,
                               int32_t* M) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t m = mate[v];
    const int64_t rep = (m >= 0 && (int64_t)m < v) ? m : v;
    M[v] = rank[rep];
  }
}

unsigned mgrid(const Ctx& c, int64_t items_per_block, int64_t n) {
  int64_t g = (n + items_per_block - 1) / items_per_block;
  const int64_t cap = (int64_t)c.num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

int bits_of(int64_t x) {  // smallest b with x < 2^b
  int b = 0;
  while (b < 62 && (1LL << b) <= x) b++;
  return b;
}

int64_t read_count(Ctx& c, const int64_t* d) {
  GM_CUDA(cudaMemcpyAsync(c.h_small, d, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  return c.h_small[0];
}

}  // namespace

// Matches level lvl and writes its map to the next level into L.M; returns
// n_c.  Uses the clustering scratch (labels as partners, requests as
// preferences, the rank array) and the sort buffers.
int32_t match_level(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  const int32_t n = L.n;
  const MatchGraph g{n, L.xadj, L.adj, L.adjw, L.vw};
  int32_t* mate = c.C;
  int32_t* pref = c.req;
  int64_t* ctr = c.counters + 6;     // matched in a round; keys of a stage
  int64_t* got = c.counters + 7;     // matched in a stage
  GM_CUDA(cudaMemsetAsync(mate, 0xFF, (size_t)std::max(1, n) * sizeof(int32_t), c.st));  // -1
  const unsigned gs = mgrid(c, kMThreads / kSubWarp, n), gv = mgrid(c, kMThreads, n);
  int64_t matched = 0;
  for (int32_t r = 0; r < c.cfg.match_rounds; r++) {
    GM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(int64_t), c.st));
    k_match_prefer<<<gs, kMThreads, 0, c.st>>>(g, mate, c.lmax, c.cfg.seed, lvl, pref); count_launch();
    k_match_mutual<<<gv, kMThreads, 0, c.st>>>(n, pref, mate, ctr); count_launch();
    const int64_t now = read_count(c, ctr);
    matched += now;
    if (now == 0) break;
  }
  const int idbits = bits_of(n);
  for (int stage = 1; stage <= 4; stage++) {
    if (4 * matched > 3 * (int64_t)n) break;
    // group bits: a vertex id (leaves, relatives), 31 hash bits (twins), none (isolated)
    const int gbits = stage == 2 ? 31 : stage == 4 ? 0 : idbits;
    GM_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(int64_t), c.st));
    k_twohop_keys<<<gv, kMThreads, 0, c.st>>>(g, mate, stage, c.cfg.seed, idbits, c.sort.key[0], c.sort.val[0],
                                             ctr); count_launch();
    const int cur = radix_sort_pairs(c.sort, n, ctr, std::max(1, gbits + idbits), c.st);
    k_pair_groups<<<gv, kMThreads, 0, c.st>>>(c.sort.key[cur], c.sort.val[cur], ctr, idbits, g, c.lmax,
                                             stage == 2 ? 1 : 0, mate, got); count_launch();
    matched += read_count(c, got);
  }
  // number pairs and singles by their smallest member
  scan(LoadRep{mate}, StoreRank{c.rank}, n, nullptr, c.scan, c.st);
  const int64_t nc = read_count(c, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(n)));
  if (!L.M) L.M = c.mem.make<int32_t>((size_t)std::max(1, n));
  k_match_number<<<gv, kMThreads, 0, c.st>>>(n, mate, c.rank, L.M); count_launch();
  GM_CUDA(cudaGetLastError());
  return (int32_t)nc;
}

}  // namespace gm
