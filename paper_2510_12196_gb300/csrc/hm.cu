// Hierarchical multisection (GPU-HM, Section 4.1 "Hierarchical
// Multisection": Eq. 2, Alg. 2, Alg. 3).
//
// The recursion of Alg. 3 runs breadth first over the hierarchy: all
// subgraphs of one level sit stacked in one set of arrays (subgraph j's
// vertices at [voff_j, voff_{j+1}), its entries at [eoff_j, eoff_{j+1}),
// its local row pointers at voff_j + j).  Each is partitioned into a_i
// blocks by the library's own multilevel pipeline on the one-level hierarchy
// a_i with distance 1 (J = 2 * edge cut) under Eq. 2's adaptive imbalance;
// the partitions are independent, so a pool of host threads runs them on
// their own streams.  The a_i children of every subgraph are then built at
// once on the device (Alg. 2 for all blocks of all subgraphs together): a
// radix sort of (child, vertex) gives each child's members in ascending id,
// a scan of the in-block degrees gives the row pointers, and one pass copies
// the in-block entries in adjacency order with the children's local ids.
// The result equals Alg. 2 run block by block.  Block b at level i adds
// b * a_1 ... a_{i-1} to the PE id (a_1 varies fastest).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"

namespace gm {
namespace {

constexpr int kHThreads = 256;

// the subgraphs of one hierarchy level, stacked
struct Stack {
  int32_t cnt = 0;
  std::vector<int64_t> voff, eoff;  // host, cnt + 1
  std::vector<int64_t> weight;      // host, c(V') per subgraph
  int64_t* X = nullptr;      // n + cnt local row pointers
  int32_t* A = nullptr;      // entries (local ids)
  int32_t* W = nullptr;      // entry weights
  int32_t* VW = nullptr;     // [n] vertex weights
  int32_t* ORIG = nullptr;   // [n] vertex of the input graph
  int32_t* BASE = nullptr;   // [n] PE id contributed by the levels above
  int32_t* SUB = nullptr;    // [n] subgraph index
  int64_t* VOFF = nullptr;   // [cnt + 1] device copy of voff
  int64_t* EOFF = nullptr;   // [cnt + 1] device copy of eoff
  bool owns_graph = true;    // X, A, W, VW allocated here (not the input level's)
};

unsigned hgrid(const Ctx& c, int64_t n) {
  int64_t g = (n + kHThreads - 1) / kHThreads;
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

__global__ void k_hm_init(int32_t n, int32_t* orig, int32_t* base, int32_t* sub) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    orig[v] = (int32_t)v;
    base[v] = 0;
    sub[v] = 0;
  }
}

// a partitioner's result (PE codes of the one-level hierarchy) as block ids
__global__ void k_hm_take(int32_t n, const int32_t* __restrict__ codes, const int32_t* __restrict__ pe_of_code,
                          int32_t* part) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    part[v] = pe_of_code[codes[v]];
}

// keys (child, vertex) with child = subgraph * a + block
__global__ void k_hm_keys(int32_t n, const int32_t* __restrict__ sub, const int32_t* __restrict__ part, int32_t a,
                          int sbits, uint64_t* key, int32_t* val) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t ch = (uint64_t)sub[s] * (uint64_t)a + (uint64_t)part[s];
    key[s] = (ch << sbits) | (uint64_t)s;
    val[s] = (int32_t)s;
  }
}

// position of every vertex in the sorted order, and each child's member range
__global__ void k_hm_bounds(int32_t n, const uint64_t* __restrict__ key, const int32_t* __restrict__ val, int sbits,
                            int32_t* pos, int64_t* start, int64_t* end) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    pos[val[p]] = (int32_t)p;
    const uint64_t ch = key[p] >> sbits;
    if (p == 0 || (key[p - 1] >> sbits) != ch) start[ch] = p;
    if (p == n - 1 || (key[p + 1] >> sbits) != ch) end[ch] = p + 1;
  }
}

// in-block degree of every vertex, at its sorted position
__global__ void k_hm_degree(int32_t n, const int64_t* __restrict__ X, const int32_t* __restrict__ A,
                            const int32_t* __restrict__ sub, const int64_t* __restrict__ voff,
                            const int64_t* __restrict__ eoff, const int32_t* __restrict__ part,
                            const int32_t* __restrict__ pos, int64_t* deg) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = sub[s];
    const int64_t v0 = voff[j], ls = s - v0;
    const int32_t* row = A + eoff[j];
    const int64_t b = X[v0 + j + ls], e = X[v0 + j + ls + 1];
    const int32_t ps = part[s];
    int64_t d = 0;
    for (int64_t x = b; x < e; x++) d += part[v0 + row[x]] == ps;
    deg[pos[s]] = d;
  }
}

struct LoadDeg {
  const int64_t* d;
  __device__ int64_t operator()(int64_t i) const { return d[i]; }
};
struct StoreOff {
  int64_t* out;
  __device__ void operator()(int64_t i, int64_t e, int64_t) const { out[i] = e; }
};

// entry and weight offsets of every child (its first member's prefix)
__global__ void k_hm_child_base(int64_t nchild, const int64_t* __restrict__ voffc, const int64_t* __restrict__ e2,
                                const int64_t* __restrict__ pw, int64_t* eb, int64_t* wb) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= nchild;
       c += (int64_t)gridDim.x * blockDim.x) {
    eb[c] = e2[voffc[c]];
    wb[c] = pw[voffc[c]];
  }
}

struct LoadSortedVw {
  const int32_t* vw;
  const int32_t* val;
  __device__ int64_t operator()(int64_t p) const { return vw[val[p]]; }
};

// the children's arrays: in-block entries in adjacency order with local ids
__global__ void k_hm_fill(int32_t n, const int64_t* __restrict__ X, const int32_t* __restrict__ A,
                          const int32_t* __restrict__ W, const int32_t* __restrict__ VW,
                          const int32_t* __restrict__ ORIG, const int32_t* __restrict__ BASE,
                          const int32_t* __restrict__ sub, const int64_t* __restrict__ voff,
                          const int64_t* __restrict__ eoff, const int32_t* __restrict__ part, int32_t a,
                          int64_t below, const int32_t* __restrict__ pos, const int64_t* __restrict__ e2,
                          const int64_t* __restrict__ voffc, const int64_t* __restrict__ eb, int64_t* X2, int32_t* A2,
                          int32_t* W2, int32_t* VW2, int32_t* ORIG2, int32_t* BASE2, int32_t* SUB2) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = sub[s];
    const int64_t v0 = voff[j], ls = s - v0;
    const int32_t* row = A + eoff[j];
    const int32_t* wrow = W + eoff[j];
    const int64_t b = X[v0 + j + ls], e = X[v0 + j + ls + 1];
    const int32_t ps = part[s];
    const int64_t ch = (int64_t)j * a + ps;
    const int64_t p = pos[s];
    const int64_t c0 = voffc[ch];
    int64_t o = e2[p];
    for (int64_t x = b; x < e; x++) {
      const int64_t t = v0 + row[x];
      if (part[t] != ps) continue;
      A2[o] = (int32_t)(pos[t] - c0);
      W2[o] = wrow[x];
      o++;
    }
    X2[p + ch] = e2[p] - eb[ch];
    VW2[p] = VW[s];
    ORIG2[p] = ORIG[s];
    BASE2[p] = (int32_t)(BASE[s] + (int64_t)ps * below);
    SUB2[p] = (int32_t)ch;
  }
}

// the closing row pointer of every child
__global__ void k_hm_tail(int64_t nchild, const int64_t* __restrict__ voffc, const int64_t* __restrict__ eb,
                          int64_t* X2) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchild; c += (int64_t)gridDim.x * blockDim.x)
    X2[voffc[c + 1] + c] = eb[c + 1] - eb[c];
}

// the final level: PE = base + block, stored as a code at the input vertex
__global__ void k_hm_final(int32_t n, const int32_t* __restrict__ ORIG, const int32_t* __restrict__ BASE,
                           const int32_t* __restrict__ part, const int32_t* __restrict__ code_of_pe, int32_t* pi) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    pi[ORIG[s]] = code_of_pe[BASE[s] + part[s]];
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void free_stack(Ctx& c, Stack& S) {
  void* own[] = {(void*)S.ORIG, (void*)S.BASE, (void*)S.SUB, (void*)S.VOFF, (void*)S.EOFF};
  for (void* p : own)
    if (p) c.mem.put(p);
  if (S.owns_graph)
    for (void* p : {(void*)S.X, (void*)S.A, (void*)S.W, (void*)S.VW})
      if (p) c.mem.put(p);
  S = Stack{};
}

// Partitions every subgraph of S into a blocks (block ids into part).
void partition_level(Ctx& c, const Stack& S, int32_t i, int32_t a, int32_t* part, int32_t workers, HmStats* st) {
  int64_t kp = 1;
  for (int32_t j = 0; j < i; j++) kp *= c.hier[(size_t)j];
  const int32_t one = 1;
  std::atomic<int32_t> next{0};
  std::mutex mu;
  std::string err;
  map_status err_st = MAP_OK;
  std::vector<double> eps_of((size_t)S.cnt, 0.0);
  double t_create = 0, t_run = 0, t_destroy = 0;
  auto job = [&](int32_t j, cudaStream_t stream) -> bool {
    const int64_t nj = S.voff[(size_t)j + 1] - S.voff[(size_t)j];
    if (nj == 0) return true;
    // Eq. 2, clamped to [0, 1 - 1e-6]
    const double ratio = (1.0 + c.eps) * (double)kp * (double)c.cV / ((double)c.k * (double)S.weight[(size_t)j]);
    double ep = std::pow(ratio, 1.0 / (double)i) - 1.0;
    if (ep < 0.0) ep = 0.0;
    if (ep > 0.999999) ep = 0.999999;
    eps_of[(size_t)j] = ep;
    map_config cfg = c.cfg;
    cfg.alloc = nullptr;  // the partitioner contexts allocate stream-ordered themselves
    cfg.free = nullptr;
    cfg.alloc_user = nullptr;
    cfg.initial = 0;  // the partitioner starts from its breadth-first chunks
    map_ctx* sub = nullptr;
    const int64_t v0 = S.voff[(size_t)j], e0 = S.eoff[(size_t)j];
    const auto t0 = std::chrono::steady_clock::now();
    map_status r = map_create(S.X + v0 + j, S.A + e0, S.W + e0, S.VW + v0, (int32_t)nj, &a, &one, 1, ep, &cfg,
                              (void*)stream, 1, &sub);
    const auto t1 = std::chrono::steady_clock::now();
    if (r == MAP_OK) r = map_run(sub, nullptr, nullptr);
    if (r == MAP_OK) {
      Ctx& sc = sub->c;
      k_hm_take<<<hgrid(c, nj), kHThreads, 0, stream>>>((int32_t)nj, sc.lv[0].pi, sc.d_pe_of_code, part + v0);
      count_launch();
      if (cudaStreamSynchronize(stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) r = MAP_E_CUDA;
    }
    if (r != MAP_OK) {
      std::lock_guard<std::mutex> g(mu);
      if (err_st == MAP_OK) {
        err_st = r;
        err = std::string("partitioner on subgraph ") + std::to_string(j) + " of level " + std::to_string(i) + ": " +
              (sub ? map_last_error(sub) : map_last_error(nullptr));
      }
    }
    const auto t2 = std::chrono::steady_clock::now();
    if (sub) map_destroy(sub);
    {
      std::lock_guard<std::mutex> g(mu);
      t_create += std::chrono::duration<double, std::milli>(t1 - t0).count();
      t_run += std::chrono::duration<double, std::milli>(t2 - t1).count();
      t_destroy += ms_since(t2);
    }
    return r == MAP_OK;
  };
  const int32_t T = std::max(1, std::min(workers, S.cnt));
  if (T == 1) {
    GM_CUDA(cudaStreamSynchronize(c.st));
    for (int32_t j = 0; j < S.cnt; j++)
      if (!job(j, c.st)) break;
  } else {
    GM_CUDA(cudaStreamSynchronize(c.st));  // the stacked arrays are complete
    std::vector<std::thread> pool;
    for (int32_t t = 0; t < T; t++) {
      pool.emplace_back([&, t]() {
        (void)t;
        cudaStream_t stream = nullptr;
        if (cudaSetDevice(c.dev) != cudaSuccess ||
            cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
          cudaGetLastError();
          std::lock_guard<std::mutex> g(mu);
          if (err_st == MAP_OK) {
            err_st = MAP_E_CUDA;
            err = "could not create a worker stream";
          }
          return;
        }
        while (true) {
          const int32_t j = next.fetch_add(1);
          if (j >= S.cnt) break;
          {
            std::lock_guard<std::mutex> g(mu);
            if (err_st != MAP_OK) break;
          }
          if (!job(j, stream)) break;
        }
        cudaStreamDestroy(stream);
      });
    }
    for (auto& th : pool) th.join();
  }
  if (err_st != MAP_OK) throw ApiError(err_st, err);
  if (st) {
    st->ms_create += t_create;
    st->ms_run += t_run;
    st->ms_destroy += t_destroy;
    st->calls[i - 1] = 0;
    for (int32_t j = 0; j < S.cnt; j++)
      if (S.voff[(size_t)j + 1] > S.voff[(size_t)j]) {
        if (st->calls[i - 1] == 0) st->first_eps[i - 1] = eps_of[(size_t)j];
        st->calls[i - 1]++;
      }
  }
}

// Builds the a children of every subgraph of S (Alg. 2 for all blocks at once).
Stack build_children(Ctx& c, int32_t n, const Stack& S, int32_t i, int32_t a, const int32_t* part) {
  const int64_t nchild = (int64_t)S.cnt * a;
  int64_t below = 1;
  for (int32_t j = 0; j + 1 < i; j++) below *= c.hier[(size_t)j];
  const unsigned gv = hgrid(c, n);
  const int sbits = bits_of(n);
  const int cbits = bits_of(nchild);
  // members of every child in ascending id
  k_hm_keys<<<gv, kHThreads, 0, c.st>>>(n, S.SUB, part, a, sbits, c.sort.key[0], c.sort.val[0]); count_launch();
  const int cur = radix_sort_pairs(c.sort, n, nullptr, sbits + std::max(1, cbits), c.st);
  int64_t* start = c.mem.make<int64_t>((size_t)nchild);
  int64_t* end = c.mem.make<int64_t>((size_t)nchild);
  GM_CUDA(cudaMemsetAsync(start, 0, (size_t)nchild * sizeof(int64_t), c.st));
  GM_CUDA(cudaMemsetAsync(end, 0, (size_t)nchild * sizeof(int64_t), c.st));
  int32_t* pos = c.rank;
  k_hm_bounds<<<gv, kHThreads, 0, c.st>>>(n, c.sort.key[cur], c.sort.val[cur], sbits, pos, start, end); count_launch();
  std::vector<int64_t> hs((size_t)nchild), he((size_t)nchild);
  GM_CUDA(cudaMemcpyAsync(hs.data(), start, (size_t)nchild * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(he.data(), end, (size_t)nchild * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  Stack C;
  C.cnt = (int32_t)nchild;
  C.voff.assign((size_t)nchild + 1, 0);
  for (int64_t ch = 0; ch < nchild; ch++) C.voff[(size_t)ch + 1] = C.voff[(size_t)ch] + (he[(size_t)ch] - hs[(size_t)ch]);
  if (C.voff[(size_t)nchild] != n) throw ApiError(MAP_E_INTERNAL, "hierarchical multisection: child sizes do not add up");
  C.VOFF = c.mem.make<int64_t>((size_t)nchild + 1);
  GM_CUDA(cudaMemcpyAsync(C.VOFF, C.voff.data(), ((size_t)nchild + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.st));
  // in-block degrees at the sorted positions, their prefix = entry offsets
  int64_t* deg = c.gain;
  k_hm_degree<<<gv, kHThreads, 0, c.st>>>(n, S.X, S.A, S.SUB, S.VOFF, S.EOFF, part, pos, deg); count_launch();
  int64_t* e2 = c.P64;
  scan(LoadDeg{deg}, StoreOff{e2}, n, nullptr, c.scan, c.st);
  GM_CUDA(cudaMemcpyAsync(e2 + n, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(n)), sizeof(int64_t),
                          cudaMemcpyDeviceToDevice, c.st));
  int64_t* pw = c.P64b;
  scan(LoadSortedVw{S.VW, c.sort.val[cur]}, StoreOff{pw}, n, nullptr, c.scan, c.st);
  GM_CUDA(cudaMemcpyAsync(pw + n, c.scan.tile_sums + std::max<int64_t>(1, scan_tiles(n)), sizeof(int64_t),
                          cudaMemcpyDeviceToDevice, c.st));
  int64_t* eb = c.mem.make<int64_t>((size_t)nchild + 1);
  int64_t* wb = c.mem.make<int64_t>((size_t)nchild + 1);
  k_hm_child_base<<<hgrid(c, nchild + 1), kHThreads, 0, c.st>>>(nchild, C.VOFF, e2, pw, eb, wb); count_launch();
  std::vector<int64_t> heb((size_t)nchild + 1), hwb((size_t)nchild + 1);
  GM_CUDA(cudaMemcpyAsync(heb.data(), eb, ((size_t)nchild + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaMemcpyAsync(hwb.data(), wb, ((size_t)nchild + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
  GM_CUDA(cudaStreamSynchronize(c.st));
  C.eoff = heb;
  C.weight.assign((size_t)nchild, 0);
  for (int64_t ch = 0; ch < nchild; ch++) C.weight[(size_t)ch] = hwb[(size_t)ch + 1] - hwb[(size_t)ch];
  const int64_t m2 = heb[(size_t)nchild];
  C.EOFF = eb;
  C.X = c.mem.make<int64_t>((size_t)n + (size_t)nchild);
  C.A = c.mem.make<int32_t>((size_t)std::max<int64_t>(1, m2));
  C.W = c.mem.make<int32_t>((size_t)std::max<int64_t>(1, m2));
  C.VW = c.mem.make<int32_t>((size_t)n);
  C.ORIG = c.mem.make<int32_t>((size_t)n);
  C.BASE = c.mem.make<int32_t>((size_t)n);
  C.SUB = c.mem.make<int32_t>((size_t)n);
  k_hm_fill<<<gv, kHThreads, 0, c.st>>>(n, S.X, S.A, S.W, S.VW, S.ORIG, S.BASE, S.SUB, S.VOFF, S.EOFF, part, a, below,
                                        pos, e2, C.VOFF, eb, C.X, C.A, C.W, C.VW, C.ORIG, C.BASE, C.SUB);
  count_launch();
  k_hm_tail<<<hgrid(c, nchild), kHThreads, 0, c.st>>>(nchild, C.VOFF, eb, C.X); count_launch();
  GM_CUDA(cudaGetLastError());
  c.mem.put(start);
  c.mem.put(end);
  c.mem.put(wb);
  return C;
}

}  // namespace

void hm_run(Ctx& c, int lvl, int32_t workers, HmStats* st) {
  const auto t0 = std::chrono::steady_clock::now();
  const int32_t levels = (int32_t)c.hier.size();
  if (levels > 16) throw ApiError(MAP_E_INVALID, "hierarchical multisection supports at most 16 levels");
  if (st) {
    *st = HmStats{};
    st->levels = levels;
    st->workers = workers;
  }
  Level& L0 = c.lv[(size_t)lvl];
  const int32_t n = L0.n;
  Stack S;
  S.cnt = 1;
  S.voff = {0, (int64_t)n};
  S.eoff = {0, L0.m};
  S.weight = {c.cV};
  S.X = L0.xadj;
  S.A = L0.adj;
  S.W = L0.adjw;
  S.VW = L0.vw;
  S.owns_graph = false;
  S.ORIG = c.mem.make<int32_t>((size_t)n);
  S.BASE = c.mem.make<int32_t>((size_t)n);
  S.SUB = c.mem.make<int32_t>((size_t)n);
  S.VOFF = c.mem.make<int64_t>(2);
  S.EOFF = c.mem.make<int64_t>(2);
  GM_CUDA(cudaMemcpyAsync(S.VOFF, S.voff.data(), 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c.st));
  GM_CUDA(cudaMemcpyAsync(S.EOFF, S.eoff.data(), 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c.st));
  k_hm_init<<<hgrid(c, n), kHThreads, 0, c.st>>>(n, S.ORIG, S.BASE, S.SUB); count_launch();
  int32_t* part = c.pp;
  try {
    for (int32_t i = levels; i >= 1; i--) {
      const int32_t a = c.hier[(size_t)i - 1];
      auto tp = std::chrono::steady_clock::now();
      partition_level(c, S, i, a, part, workers, st);
      if (st) {
        st->ms_level[i - 1] = ms_since(tp);
        st->ms_partition += st->ms_level[i - 1];
      }
      if (i == 1) {
        k_hm_final<<<hgrid(c, n), kHThreads, 0, c.st>>>(n, S.ORIG, S.BASE, part, c.d_code_of_pe, L0.pi); count_launch();
        GM_CUDA(cudaGetLastError());
        break;
      }
      auto tb = std::chrono::steady_clock::now();
      Stack C = build_children(c, n, S, i, a, part);
      free_stack(c, S);
      S = C;
      GM_CUDA(cudaStreamSynchronize(c.st));
      if (st) st->ms_build += ms_since(tb);
    }
  } catch (...) {
    free_stack(c, S);
    throw;
  }
  free_stack(c, S);
  GM_CUDA(cudaStreamSynchronize(c.st));
  if (st) st->ms_total = ms_since(t0);
}

}  // namespace gm
