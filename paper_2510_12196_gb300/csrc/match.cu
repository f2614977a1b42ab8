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

// Compares the exp*2 ratings ww1 / c1 and ww2 / c2 (ww = w^2) exactly:
// ww1 c2 against ww2 c1 in 128 bits; -1, 0 or 1.
__device__ __forceinline__ int rating_cmp(uint64_t ww1, uint64_t c1, uint64_t ww2, uint64_t c2) {
  if (c1 == c2) return ww1 == ww2 ? 0 : (ww1 > ww2 ? 1 : -1);
  const uint64_t lo1 = ww1 * c2, hi1 = __umul64hi(ww1, c2);
  const uint64_t lo2 = ww2 * c1, hi2 = __umul64hi(ww2, c1);
  if (hi1 != hi2) return hi1 > hi2 ? 1 : -1;
  return lo1 == lo2 ? 0 : (lo1 > lo2 ? 1 : -1);
}

// A vertex's best candidate so far: rating ww / c, the neighbour u and the
// noise hash of the edge (computed on the first tie only).
struct Pref {
  uint64_t ww, c, h;
  int32_t u;
  bool hk;
};

// Offers neighbour (ww, c, u) of v: larger rating, then smaller edge hash,
// then smaller u.
__device__ __forceinline__ void pref_offer(Pref& b, uint64_t ww, uint64_t c, int32_t u, int32_t v, uint64_t seed,
                                           int32_t level) {
  if (b.u < 0) {
    b = Pref{ww, c, 0, u, false};
    return;
  }
  const int r = rating_cmp(ww, c, b.ww, b.c);
  if (r > 0) {
    b = Pref{ww, c, 0, u, false};
    return;
  }
  if (r < 0) return;
  if (!b.hk) {
    b.h = h_edge(seed, level, min(v, b.u), max(v, b.u));
    b.hk = true;
  }
  const uint64_t hu = h_edge(seed, level, min(v, u), max(v, u));
  if (hu < b.h || (hu == b.h && u < b.u)) b = Pref{ww, c, hu, u, true};
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
    Pref b{0, 0, 0, -1, false};
    if (free_v) {
      const int64_t cv = g.vw[v];
      for (int64_t x = g.xadj[v] + sl; x < g.xadj[v + 1]; x += kSubWarp) {
        const int32_t u = g.adj[x];
        if (mate[u] >= 0) continue;
        const int64_t cu = g.vw[u];
        if (cv + cu > lmax) continue;
        const uint64_t w = (uint64_t)g.adjw[x];
        pref_offer(b, w * w, (uint64_t)cu, u, v, seed, level);
      }
      if (b.u >= 0 && !b.hk) b.h = h_edge(seed, level, min(v, b.u), max(v, b.u));
    }
    // sub-warp reduction on (rating, hash, u), hashes known
#pragma unroll
    for (int o = kSubWarp / 2; o > 0; o >>= 1) {
      const uint64_t oww = __shfl_xor_sync(0xffffffffu, b.ww, o);
      const uint64_t oc = __shfl_xor_sync(0xffffffffu, b.c, o);
      const uint64_t oh = __shfl_xor_sync(0xffffffffu, b.h, o);
      const int32_t ou = __shfl_xor_sync(0xffffffffu, b.u, o);
      if (ou < 0) continue;
      bool take = b.u < 0;
      if (!take) {
        const int r = rating_cmp(oww, oc, b.ww, b.c);
        take = r > 0 || (r == 0 && (oh < b.h || (oh == b.h && ou < b.u)));
      }
      if (take) b = Pref{oww, oc, oh, ou, true};
    }
    if (sl == 0 && v0 < g.n) pref[v] = free_v ? b.u : -1;
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

// device state of one level's matching
struct MatchState {
  int64_t matched;  // vertices matched so far
  int64_t now;      // matched by the current heavy-edge round
  int64_t nkeys;    // keys of the current two-hop stage
  int64_t got;      // matched by the current two-hop stage
  int64_t nc;       // coarse vertices
  int32_t round;
  int32_t pad;
  unsigned long long kernels;  // kernels run inside conditional bodies
};

__global__ void k_mt_init(MatchState* s, int32_t rounds, cudaGraphConditionalHandle h, int use_h) {
  s->matched = 0;
  s->now = 0;
  s->round = 0;
  s->kernels = 0;
  if (use_h) cudaGraphSetConditional(h, rounds > 0 ? 1u : 0u);
}
__global__ void k_mt_round_end(MatchState* s, int32_t rounds, cudaGraphConditionalHandle h, int use_h,
                               unsigned long long body_kernels) {
  s->kernels += body_kernels;
  s->matched += s->now;
  s->round += 1;
  const bool more = s->now > 0 && s->round < rounds;
  s->now = 0;
  if (use_h) cudaGraphSetConditional(h, more ? 1u : 0u);
}
// a two-hop stage runs while at most 75% of the vertices are matched
__global__ void k_mt_stage_begin(MatchState* s, int32_t n, cudaGraphConditionalHandle h, int use_h) {
  s->nkeys = 0;
  s->got = 0;
  if (use_h) cudaGraphSetConditional(h, 4 * s->matched <= 3 * (int64_t)n ? 1u : 0u);
}
__global__ void k_mt_stage_end(MatchState* s, unsigned long long body_kernels) {
  s->matched += s->got;
  s->kernels += body_kernels;
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

MatchState* state_of(Ctx& c) {
  if (!c.mstate) c.mstate = c.mem.make<MatchState>(1);
  return static_cast<MatchState*>(c.mstate);
}

MatchGraph mview(const Level& L) { return MatchGraph{L.n, L.xadj, L.adj, L.adjw, L.vw}; }

// one heavy-edge round: preferences, then mutual pairs counted into s->now
void emit_round(Ctx& c, int lvl, cudaStream_t st) {
  const Level& L = c.lv[lvl];
  const int32_t n = L.n;
  c.prof_level = lvl;
  cudaEvent_t ev = c.prof_begin();
  k_match_prefer<<<mgrid(c, kMThreads / kSubWarp, n), kMThreads, 0, st>>>(mview(L), c.C, c.lmax, c.cfg.seed, lvl,
                                                                         c.req); count_launch();
  // per vertex: xadj 8, mate 4, c(v) 4, p 4; per entry: adjacency 4, weight 4, mate(u) 4, c(u) 4 (every row
  // read in full: an upper bound after the first round, when matched vertices skip theirs)
  c.prof_end(ev, PK_MATCH, 20 * (int64_t)n + 16 * L.m);
  k_match_mutual<<<mgrid(c, kMThreads, n), kMThreads, 0, st>>>(n, c.req, c.C, &state_of(c)->now); count_launch();
}

// one two-hop stage (its keys, their sort, the pairing), matched count into s->got
void emit_stage(Ctx& c, int lvl, int stage, cudaStream_t st, unsigned long long* kcount) {
  const Level& L = c.lv[lvl];
  const int32_t n = L.n;
  MatchState* s = state_of(c);
  const int idbits = bits_of(n);
  // group bits: a vertex id (leaves, relatives), 31 hash bits (twins), none (isolated)
  const int gbits = stage == 2 ? 31 : stage == 4 ? 0 : idbits;
  const unsigned gv = mgrid(c, kMThreads, n);
  k_twohop_keys<<<gv, kMThreads, 0, st>>>(mview(L), c.C, stage, c.cfg.seed, idbits, c.sort.key[0], c.sort.val[0],
                                          &s->nkeys); count_launch();
  const int cur = radix_sort_pairs(c.sort, n, &s->nkeys, std::max(1, gbits + idbits), st,
                                   kcount ? &c.cap : nullptr, kcount);
  k_pair_groups<<<gv, kMThreads, 0, st>>>(c.sort.key[cur], c.sort.val[cur], &s->nkeys, idbits, mview(L), c.lmax,
                                          stage == 2 ? 1 : 0, c.C, &s->got); count_launch();
}

// pairs and single vertices numbered by their smallest member into L.M
void emit_number(Ctx& c, int lvl, cudaStream_t st) {
  Level& L = c.lv[lvl];
  const int32_t n = L.n;
  scan(LoadRep{c.C}, StoreRank{c.rank}, n, nullptr, c.scan, st);
  GM_CUDA(cudaMemcpyAsync(&state_of(c)->nc, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(n)),
                          sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  k_match_number<<<mgrid(c, kMThreads, n), kMThreads, 0, st>>>(n, c.C, c.rank, L.M); count_launch();
}

// Captures the matching of one level: rounds in a WHILE node, each two-hop
// stage in an IF node on the 75% rule, then the numbering.
void build_match_graph(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  if (L.cgexec) cudaGraphExecDestroy(L.cgexec);
  L.cgexec = nullptr;
  MatchState* s = state_of(c);
  cudaStream_t saved = c.st;
  cap_streams(c);
  cudaStream_t cs = c.cap.s[0];
  long long root = 0, body = 0;
  long long* outer = set_capture_counter(&root);
  GM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  c.cap.depth = 0;
  c.st = cs;
  try {
    GM_CUDA(cudaMemsetAsync(c.C, 0xFF, (size_t)std::max(1, L.n) * sizeof(int32_t), cs));  // mate = -1
    cudaGraphConditionalHandle h = cap_handle(cs, 0);
    k_mt_init<<<1, 1, 0, cs>>>(s, c.cfg.match_rounds, h, 1); count_launch();
    cap_cond(c.cap, cs, h, cudaGraphCondTypeWhile, [&](cudaStream_t bs) {
      body = 0;
      set_capture_counter(&body);
      emit_round(c, lvl, bs);
      k_mt_round_end<<<1, 1, 0, bs>>>(s, c.cfg.match_rounds, h, 1, (unsigned long long)body + 1); count_launch();
      set_capture_counter(&root);
    });
    for (int stage = 1; stage <= 4; stage++) {
      cudaGraphConditionalHandle hs = cap_handle(cs, 0);
      k_mt_stage_begin<<<1, 1, 0, cs>>>(s, L.n, hs, 1); count_launch();
      cap_cond(c.cap, cs, hs, cudaGraphCondTypeIf, [&](cudaStream_t bs) {
        body = 0;
        set_capture_counter(&body);
        emit_stage(c, lvl, stage, bs, &s->kernels);
        k_mt_stage_end<<<1, 1, 0, bs>>>(s, (unsigned long long)body + 1); count_launch();
        set_capture_counter(&root);
      });
    }
    emit_number(c, lvl, cs);
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

}  // namespace

// Matches level lvl and writes its map to the next level into L.M; returns
// n_c.  Uses the clustering scratch (labels as partners, requests as
// preferences, the rank array) and the sort buffers.
int32_t match_level(Ctx& c, int lvl) {
  Level& L = c.lv[lvl];
  const int32_t n = L.n;
  MatchState* s = state_of(c);
  if (!L.M) L.M = c.mem.make<int32_t>((size_t)std::max(1, n));
  if (c.use_graphs && !c.prof) {
    // the graph writes L.M, which a stalled level gives back, so its address is part of the key
    const int64_t key[6] = {(int64_t)n, L.m, c.lmax, (int64_t)c.cfg.match_rounds, -1, (int64_t)(intptr_t)L.M};
    bool same = L.cgexec != nullptr;
    for (int i = 0; i < 6 && same; i++) same = L.cg_key[i] == key[i];
    if (!same) {
      build_match_graph(c, lvl);
      for (int i = 0; i < 6; i++) L.cg_key[i] = key[i];
    }
    GM_CUDA(cudaGraphLaunch(L.cgexec, c.st));
    GM_CUDA(cudaMemcpyAsync(c.h_small, &s->nc, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
    GM_CUDA(cudaMemcpyAsync(c.h_small + 1, &s->kernels, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
    GM_CUDA(cudaStreamSynchronize(c.st));
    add_launches(L.cg_root + (long long)c.h_small[1]);
    return (int32_t)c.h_small[0];
  }
  // stream launches: the same kernels, the loop decisions taken on the host
  auto read = [&](const int64_t* d) {
    GM_CUDA(cudaMemcpyAsync(c.h_small, d, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
    GM_CUDA(cudaStreamSynchronize(c.st));
    return c.h_small[0];
  };
  GM_CUDA(cudaMemsetAsync(c.C, 0xFF, (size_t)std::max(1, n) * sizeof(int32_t), c.st));
  k_mt_init<<<1, 1, 0, c.st>>>(s, c.cfg.match_rounds, 0, 0); count_launch();
  for (int32_t r = 0; r < c.cfg.match_rounds; r++) {
    emit_round(c, lvl, c.st);
    const int64_t now = read(&s->now);
    k_mt_round_end<<<1, 1, 0, c.st>>>(s, c.cfg.match_rounds, 0, 0, 0); count_launch();
    if (now == 0) break;
  }
  for (int stage = 1; stage <= 4; stage++) {
    k_mt_stage_begin<<<1, 1, 0, c.st>>>(s, n, 0, 0); count_launch();
    if (4 * read(&s->matched) > 3 * (int64_t)n) break;
    emit_stage(c, lvl, stage, c.st, nullptr);
    k_mt_stage_end<<<1, 1, 0, c.st>>>(s, 0); count_launch();
  }
  emit_number(c, lvl, c.st);
  GM_CUDA(cudaGetLastError());
  return (int32_t)read(&s->nc);
}

}  // namespace gm
