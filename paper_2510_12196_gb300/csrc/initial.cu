// Initial mapping of a large coarsest graph with the whole GPU.
//
// The mapping is the breadth-first one of the single-CTA kernel (and of the
// oracle): vertices in the order of a FIFO breadth-first search that starts
// at the lowest unvisited id whenever the queue runs empty, neighbours taken
// in adjacency order; the vertex with preceding weight s goes to PE
// floor(s k / c(V)).  That order is produced here without a queue:
//   1. connected components, each labelled by its smallest id: hooking of the
//      larger label onto the smaller one along each vertex's first and then
//      second edge, with pointer jumping after each pass; then, with the most
//      frequent label among sampled vertices taken as the giant component's,
//      hooking along every edge of the vertices outside it, and jumping,
//      until no such edge joins two labels (an edge between the giant and
//      another vertex is seen from the other side, so then no edge at all
//      joins two labels; labels only ever move to smaller ones, so each ends
//      as its component's smallest id);
//   2. one level-synchronous search from all component roots at once: the
//      frontier is kept in order, every unvisited neighbour is claimed by its
//      earliest frontier vertex, and the children are laid out by a scan over
//      the frontier's (vertex, adjacency index) slots, which is exactly the
//      order a FIFO queue appends them in;
//   3. a sort by (component label, position in the layered order), which puts
//      each component's search order after the components with smaller ids.
// Coarsest graphs small enough for shared memory keep the one-CTA kernel.
#include <algorithm>

#include "engine.h"

namespace gm {
namespace {

constexpr int kIThreads = 256;

unsigned igrid(const Ctx& c, int64_t n) {
  int64_t g = (n + kIThreads - 1) / kIThreads;
  const int64_t cap = (int64_t)c.num_sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

int bits_of(int64_t x) {  // smallest b with x < 2^b
  int b = 0;
  while (b < 62 && (1LL << b) <= x) b++;
  return b;
}

__global__ void k_cc_init(int32_t n, int32_t* lab, int32_t* lev, int32_t* claim) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    lab[v] = (int32_t)v;
    lev[v] = -1;
    claim[v] = INT32_MAX;
  }
}

// hooking along the r-th edge of every vertex (sampling passes)
__global__ void k_cc_sample(int32_t n, const int64_t* __restrict__ xadj, const int32_t* __restrict__ adj, int32_t* lab,
                            int32_t r) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = xadj[v] + r;
    if (e >= xadj[v + 1]) continue;
    const int32_t lu = lab[v], lv = lab[adj[e]];
    if (lu != lv) atomicMin(&lab[max(lu, lv)], min(lu, lv));
  }
}

// hooking along every edge of the vertices whose label is not `giant` (one
// warp per vertex)
__global__ void k_cc_hook_rest(int32_t n, const int64_t* __restrict__ xadj, const int32_t* __restrict__ adj,
                               int32_t* lab, int32_t giant, int32_t* changed) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool any = false;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    if (__shfl_sync(0xffffffffu, lab[u], 0) == giant) continue;
    for (int64_t e = xadj[u] + lane; e < xadj[u + 1]; e += 32) {
      const int32_t lu = lab[u], lv = lab[adj[e]];
      if (lu == lv) continue;
      atomicMin(&lab[max(lu, lv)], min(lu, lv));
      any = true;
    }
  }
  if (__any_sync(0xffffffffu, any) && lane == 0) *changed = 1;
}

// the labels of kCcSample spread vertices (to find the giant component's)
constexpr int kCcSample = 1024;
__global__ void k_cc_pick(int32_t n, const int32_t* __restrict__ lab, int32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kCcSample) out[i] = lab[(int64_t)(((uint64_t)i * 2654435761ULL) % (uint64_t)n)];
}

// pointer jumping with path halving: every label becomes the root of its
// chain; the halving shortens the chains the other threads walk (labels only
// decrease, so every chain has fewer than n steps)
__global__ void k_cc_jump(int32_t n, int32_t* lab, uint32_t* err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = (int32_t)v;
    bool done = false;
    for (int32_t step = 0; step < n; step++) {
      const int32_t p = lab[x];
      if (p == x) {
        done = true;
        break;
      }
      const int32_t gp = lab[p];
      if (gp != p) atomicMin(&lab[x], gp);
      x = gp;
    }
    if (!done) atomicOr(err, ERR_TIMEOUT);
    atomicMin(&lab[v], x);
  }
}

// component roots (label = own id), ascending
struct LoadRoot {
  const int32_t* lab;
  __device__ int64_t operator()(int64_t v) const { return lab[v] == (int32_t)v ? 1 : 0; }
};
struct StoreRoot {
  int32_t* order;
  int32_t* lev;
  __device__ void operator()(int64_t v, int64_t e, int64_t x) const {
    if (!x) return;
    order[e] = (int32_t)v;
    lev[v] = 0;
  }
};

// degrees of the frontier vertices (their slots)
struct LoadFrontierDeg {
  const int32_t* order;
  const int64_t* xadj;
  int64_t head;
  __device__ int64_t operator()(int64_t i) const {
    const int32_t u = order[head + i];
    return xadj[u + 1] - xadj[u];
  }
};
struct StoreOffs {
  int64_t* out;
  __device__ void operator()(int64_t i, int64_t e, int64_t) const { out[i] = e; }
};

// slot s of the frontier: its frontier index i (offs[i] <= s < offs[i + 1])
__device__ __forceinline__ int64_t slot_owner(const int64_t* offs, int64_t F, int64_t s) {
  int64_t lo = 0, hi = F;  // offs[lo] <= s < offs[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (offs[mid] <= s) lo = mid;
    else hi = mid;
  }
  return lo;
}

struct Frontier {
  const int32_t* order;
  const int64_t* xadj;
  const int32_t* adj;
  const int64_t* offs;
  int64_t head, F;
  // the neighbour of slot s and its frontier index
  __device__ __forceinline__ int32_t at(int64_t s, int64_t& i) const {
    i = slot_owner(offs, F, s);
    const int32_t u = order[head + i];
    return adj[xadj[u] + (s - offs[i])];
  }
};

__global__ void k_bfs_claim(Frontier f, int64_t S, const int32_t* __restrict__ lev, int32_t* claim) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    const int32_t w = f.at(s, i);
    if (lev[w] < 0) atomicMin(&claim[w], (int32_t)i);
  }
}

// slot s appends its neighbour iff the neighbour is unvisited and this
// frontier vertex claimed it first
struct LoadChild {
  Frontier f;
  const int32_t* lev;
  const int32_t* claim;
  __device__ int64_t operator()(int64_t s) const {
    int64_t i;
    const int32_t w = f.at(s, i);
    return (lev[w] < 0 && claim[w] == (int32_t)i) ? 1 : 0;
  }
};

__global__ void k_bfs_write(Frontier f, int64_t S, const int64_t* __restrict__ pos, int64_t tail, int32_t level,
                            const int32_t* __restrict__ claim, int32_t* lev, int32_t* order) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    const int32_t w = f.at(s, i);
    // only the claiming slot writes lev[w], so its test is not raced
    if (lev[w] < 0 && claim[w] == (int32_t)i) {
      order[tail + pos[s]] = w;
      lev[w] = level;
    }
  }
}

// sort keys: (component label, position in the layered order)
__global__ void k_order_keys(int32_t n, const int32_t* __restrict__ order, const int32_t* __restrict__ lab,
                             uint64_t* key, int32_t* val) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = order[p];
    key[p] = ((uint64_t)(uint32_t)lab[v] << 32) | (uint64_t)p;
    val[p] = v;
  }
}

struct LoadOrderedVw {
  const int32_t* val;
  const int32_t* vw;
  __device__ int64_t operator()(int64_t q) const { return vw[val[q]]; }
};
struct StorePe {
  const int32_t* val;
  const int32_t* code_of_pe;
  int64_t k, cV;
  int32_t* pi;
  __device__ void operator()(int64_t q, int64_t s, int64_t) const { pi[val[q]] = code_of_pe[(s * k) / cV]; }
};

int64_t read_dev(Ctx& c, const int64_t* d) {
  GM_CUDA(cudaMemcpyAsync(c.h_small + 6, d, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  return c.h_small[6];
}

}  // namespace

bool initial_map_large(Ctx& c) {
  Level& L = c.lv.back();
  const int32_t n = L.n;
  const int64_t m = L.m;
  int32_t* lab = c.C;
  int32_t* lev = c.Wc;
  int32_t* claim = c.ReqW;
  int32_t* order = c.req;
  int32_t* src = c.sort.val[1];     // free until the final sort
  int64_t* offs = c.P64b;           // frontier slot offsets (n + 1)
  int64_t* pos = c.P64;             // child positions per slot (m + 1)
  int32_t* changed = reinterpret_cast<int32_t*>(c.counters + 6);
  const unsigned gn = igrid(c, n);
  GM_CUDA(cudaMemsetAsync(c.errword, 0, sizeof(uint32_t), c.st));
  k_cc_init<<<gn, kIThreads, 0, c.st>>>(n, lab, lev, claim); count_launch();
  // 1. components labelled by their smallest id
  if (m > 0) {
    for (int32_t r = 0; r < 2; r++) {
      k_cc_sample<<<gn, kIThreads, 0, c.st>>>(n, L.xadj, L.adj, lab, r); count_launch();
      k_cc_jump<<<gn, kIThreads, 0, c.st>>>(n, lab, c.errword); count_launch();
    }
    // the most frequent sampled label: the giant component's, if there is one
    int32_t* picks = src;
    k_cc_pick<<<(kCcSample + kIThreads - 1) / kIThreads, kIThreads, 0, c.st>>>(n, lab, picks); count_launch();
    std::vector<int32_t> h(kCcSample);
    GM_CUDA(cudaMemcpyAsync(h.data(), picks, kCcSample * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    GM_CUDA(cudaStreamSynchronize(c.st));
    std::sort(h.begin(), h.end());
    int32_t giant = h[0], best = 0;
    for (int i = 0; i < kCcSample;) {
      int j = i;
      while (j < kCcSample && h[j] == h[i]) j++;
      if (j - i > best) {
        best = j - i;
        giant = h[i];
      }
      i = j;
    }
    for (int it = 0;; it++) {
      if (it > 64 + 4 * bits_of(n)) return false;  // not settled: the caller takes the one-CTA search
      GM_CUDA(cudaMemsetAsync(changed, 0, sizeof(int64_t), c.st));
      k_cc_hook_rest<<<igrid(c, (int64_t)n * 32), kIThreads, 0, c.st>>>(n, L.xadj, L.adj, lab, giant, changed);
      count_launch();
      k_cc_jump<<<gn, kIThreads, 0, c.st>>>(n, lab, c.errword); count_launch();
      if (read_dev(c, c.counters + 6) == 0) break;
    }
  }
  // 2. the layered search from every root at once
  scan(LoadRoot{lab}, StoreRoot{order, lev}, n, nullptr, c.scan, c.st);
  int64_t head = 0, tail = read_dev(c, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(n)));
  for (int32_t level = 1; head < tail; level++) {
    if (level > n) throw ApiError(MAP_E_INTERNAL, "breadth-first search did not end");
    const int64_t F = tail - head;
    scan(LoadFrontierDeg{order, L.xadj, head}, StoreOffs{offs}, F, nullptr, c.scan, c.st);
    GM_CUDA(cudaMemcpyAsync(offs + F, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(F)), sizeof(int64_t),
                            cudaMemcpyDeviceToDevice, c.st));
    const int64_t S = read_dev(c, offs + F);
    if (S == 0) {  // no edges leave this frontier
      head = tail;
      continue;
    }
    const Frontier f{order, L.xadj, L.adj, offs, head, F};
    const unsigned gs = igrid(c, S);
    k_bfs_claim<<<gs, kIThreads, 0, c.st>>>(f, S, lev, claim); count_launch();
    scan(LoadChild{f, lev, claim}, StoreOffs{pos}, S, nullptr, c.scan, c.st);
    const int64_t T = read_dev(c, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(S)));
    k_bfs_write<<<gs, kIThreads, 0, c.st>>>(f, S, pos, tail, level, claim, lev, order); count_launch();
    head = tail;
    tail += T;
  }
  if (tail != n) throw ApiError(MAP_E_INTERNAL, "breadth-first search missed vertices");
  // 3. components in the order of their smallest id, each in its search order
  k_order_keys<<<gn, kIThreads, 0, c.st>>>(n, order, lab, c.sort.key[0], c.sort.val[0]); count_launch();
  const int cur = radix_sort_pairs(c.sort, n, nullptr, 32 + bits_of(n), c.st);
  scan(LoadOrderedVw{c.sort.val[cur], L.vw}, StorePe{c.sort.val[cur], c.d_code_of_pe, c.k, c.cV, L.pi}, n, nullptr,
       c.scan, c.st);
  GM_CUDA(cudaGetLastError());
  c.h_small[7] = 0;
  GM_CUDA(cudaMemcpyAsync(c.h_small + 7, c.errword, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  if (c.h_small[7] & ERR_TIMEOUT) throw ApiError(MAP_E_TIMEOUT, "a bounded device loop gave up");
  return true;
}

}  // namespace gm
