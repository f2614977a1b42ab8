// C ABI of the mapping library (declared in include/gpumap.h).  Marshals
// arguments, owns the context's device memory and converts PE ids to the
// internal PE codes; every step of the path itself runs in the kernels of
// refine.cu and coarsen.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

#include "engine.h"

namespace gm {

namespace {
std::mutex g_pin_mu;
std::vector<void*> g_pin_free;
constexpr int kPinnedSlab = 16;  // blocks per cudaMallocHost
}  // namespace

void* pinned_get(size_t bytes) {
  if (bytes > kPinnedBlock) throw std::runtime_error("pinned_get: request larger than a block");
  {
    std::lock_guard<std::mutex> g(g_pin_mu);
    if (!g_pin_free.empty()) {
      void* p = g_pin_free.back();
      g_pin_free.pop_back();
      return p;
    }
  }
  void* slab = nullptr;
  GM_CUDA(cudaMallocHost(&slab, kPinnedBlock * kPinnedSlab));
  std::lock_guard<std::mutex> g(g_pin_mu);
  for (int i = 1; i < kPinnedSlab; i++) g_pin_free.push_back(static_cast<char*>(slab) + (size_t)i * kPinnedBlock);
  return slab;
}

void pinned_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_pin_mu);
  g_pin_free.push_back(p);
}

// Stream-ordered allocations come from the device's default memory pool,
// which by default hands freed memory back to the system at every
// synchronisation, so that the next context maps it again.  Keeping up to
// kPoolKeepBytes of freed blocks in the pool makes creating and destroying
// contexts cheap (serving, hierarchical multisection, repeated maps of one
// large graph: a context for R-MAT scale 22 holds more than 8 GB, and with
// an 8 GB bound every other map_create spent about 50 ms mapping memory
// back).  Once per device.
constexpr uint64_t kPoolKeepBytes = 32ULL << 30;
void keep_pool_memory(int dev) {
  static std::atomic<unsigned long long> done{0};  // one bit per device
  const unsigned long long bit = 1ULL << (dev & 63);
  if (done.load() & bit) return;
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = kPoolKeepBytes;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
  } else {
    cudaGetLastError();
  }
  done.fetch_or(bit);
}

void* DevMem::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (afn && ffn) {
    p = afn(bytes, user, (void*)st);
    if (!p) throw ApiError(MAP_E_OOM, "allocator callback returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw ApiError(MAP_E_OOM, "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed: " +
                                    cudaGetErrorString(e));
    }
  }
  blocks.push_back({p, bytes});
  total += bytes;
  peak = std::max(peak, total);
  return p;
}

void DevMem::put(void* p) {
  for (size_t i = 0; i < blocks.size(); i++) {
    if (blocks[i].p == p) {
      if (afn && ffn) ffn(p, blocks[i].bytes, user, (void*)st);
      else cudaFreeAsync(p, st);
      total -= blocks[i].bytes;
      blocks[i] = blocks.back();
      blocks.pop_back();
      return;
    }
  }
}

void DevMem::release_all() {
  for (auto& b : blocks) {
    if (afn && ffn) ffn(b.p, b.bytes, user, (void*)st);
    else cudaFreeAsync(b.p, st);
  }
  blocks.clear();
  total = 0;
}

cudaEvent_t Ctx::prof_begin() {
  if (!prof) return nullptr;
  if (ev_used + 2 > ev_pool.size()) {
    for (int i = 0; i < 64; i++) {
      cudaEvent_t e;
      GM_CUDA(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
  }
  cudaEvent_t a = ev_pool[ev_used++];
  GM_CUDA(cudaEventRecord(a, st));
  return a;
}

void Ctx::prof_end(cudaEvent_t a, int32_t kind, int64_t bytes) {
  if (!prof || !a) return;
  cudaEvent_t b = ev_pool[ev_used++];
  GM_CUDA(cudaEventRecord(b, st));
  prof_recs.push_back(ProfRec{a, b, kind, prof_level, bytes});
}

std::string& last_create_error() {
  static thread_local std::string s;
  return s;
}

namespace {

void build_topology(Ctx& c, const int32_t* hier, const int32_t* dist, int32_t levels) {
  if (levels < 1 || levels > kMaxLevels) throw ApiError(MAP_E_INVALID, "levels must be in [1, 16]");
  Topo t{};
  t.levels = levels;
  int64_t k = 1;
  int32_t s = 0;
  t.s[0] = 0;
  for (int i = 0; i < levels; i++) {
    if (hier[i] < 1) throw ApiError(MAP_E_INVALID, "every hierarchy factor a_i must be >= 1");
    if (dist[i] < 0) throw ApiError(MAP_E_INVALID, "every distance d_i must be >= 0");
    int32_t b = 0;
    while ((1 << b) < hier[i]) b++;
    s += b;
    if (s > kMaxCodeBits) throw ApiError(MAP_E_INVALID, "PE code space exceeds 2^14 (hierarchy too large)");
    t.s[i + 1] = s;
    t.dist[i] = dist[i];
    k *= hier[i];
  }
  t.code_bits = s;
  t.kc = 1 << s;
  t.k = (int32_t)k;
  for (int b = 0; b < 32; b++) t.dist_of_bit[b] = 0;
  for (int i = 1; i <= levels; i++)
    for (int b = t.s[i - 1]; b < t.s[i]; b++) t.dist_of_bit[b] = dist[i - 1];
  c.topo = t;
  c.k = (int32_t)k;
  c.hier.assign(hier, hier + levels);
  c.dist.assign(dist, dist + levels);
  c.code_of_pe.assign((size_t)k, 0);
  c.pe_of_code.assign((size_t)t.kc, -1);
  for (int64_t p = 0; p < k; p++) {
    int64_t rem = p;
    int32_t code = 0;
    for (int i = 0; i < levels; i++) {
      const int64_t digit = rem % hier[i];
      rem /= hier[i];
      code |= (int32_t)(digit << t.s[i]);
    }
    c.code_of_pe[(size_t)p] = code;
    c.pe_of_code[(size_t)code] = (int32_t)p;
  }
}

int64_t lmax_of(int64_t total, int64_t k, double eps) {
  const double scaled = eps * 1e6;
  const int64_t e = (int64_t)(scaled < 0 ? scaled - 0.5 : scaled + 0.5);
  const int64_t num = (1000000 + e) * total;
  const int64_t den = 1000000 * k;
  return (num + den - 1) / den;
}

void alloc_sort(Ctx& c) {
  const int64_t cap = std::max<int64_t>({c.m0, (int64_t)c.n0, 1});
  c.sort.capacity = cap;
  c.sort.key[0] = c.mem.make<uint64_t>((size_t)cap);
  c.sort.key[1] = c.mem.make<uint64_t>((size_t)cap);
  c.sort.val[0] = c.mem.make<int32_t>((size_t)cap);
  c.sort.val[1] = c.mem.make<int32_t>((size_t)cap);
  const int64_t tiles = sort_tiles(cap);
  c.sort.hist = c.mem.make<int64_t>((size_t)(256 * tiles));
  c.sort.hist_off = c.mem.make<int64_t>((size_t)(256 * tiles));
  c.sort.scan.tile_sums = c.mem.make<int64_t>((size_t)(scan_tiles(256 * tiles) + 2));
  const int64_t scan_cap = std::max<int64_t>({c.m0, 2 * (int64_t)c.n0 + 2, 1});
  c.scan.tile_sums = c.mem.make<int64_t>((size_t)(scan_tiles(scan_cap) + 2));
  c.P64 = c.mem.make<int64_t>((size_t)cap + 1);
  c.P64b = c.mem.make<int64_t>((size_t)cap + 1);
}

Level& level_at(Ctx& c, int32_t level) {
  if (level < 0 || level >= (int32_t)c.lv.size())
    throw ApiError(MAP_E_STATE, "level " + std::to_string(level) + " does not exist (levels: " +
                                    std::to_string(c.lv.size()) + ")");
  return c.lv[(size_t)level];
}

template <class F>
map_status guarded(map_ctx* ctx, F&& f) {
  if (!ctx) return MAP_E_INVALID;
  try {
    ctx->c.err.clear();
    f(ctx->c);
    return MAP_OK;
  } catch (const ApiError& e) {
    ctx->c.err = e.what();
    return e.status;
  } catch (const CudaError& e) {
    ctx->c.err = e.what();
    return e.code == cudaErrorMemoryAllocation ? MAP_E_OOM : MAP_E_CUDA;
  } catch (const std::bad_alloc&) {
    ctx->c.err = "host allocation failed";
    return MAP_E_OOM;
  } catch (const std::exception& e) {
    ctx->c.err = e.what();
    return MAP_E_INTERNAL;
  }
}

void sync(Ctx& c) { GM_CUDA(cudaStreamSynchronize(c.st)); }

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace gm

using namespace gm;

extern "C" {

void map_config_default(map_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->seed = 0x5EED0000ULL;
  cfg->patience = 12;
  cfg->weak_max = 2;
  cfg->phi_num = 999;
  cfg->phi_den = 1000;
  cfg->sigma_gap = 100;
  cfg->coarsest_factor = 8;
  cfg->cluster_iters = 5;
  cfg->cluster_cap_div = 4;
  cfg->max_levels = 64;
  cfg->stall_num = 9;
  cfg->stall_den = 10;
  cfg->coarsener = 0;
  cfg->match_rounds = 16;
  cfg->initial = 0;
  cfg->lp_relax_num = 0;
  cfg->lp_relax_den = 1;
  cfg->reb_objective = 0;
  cfg->mid_deg = 0;
  cfg->split_deg = 0;
}

const char* map_status_string(map_status s) {
  switch (s) {
    case MAP_OK: return "MAP_OK";
    case MAP_E_INVALID: return "MAP_E_INVALID";
    case MAP_E_OOM: return "MAP_E_OOM";
    case MAP_E_CUDA: return "MAP_E_CUDA";
    case MAP_E_OVERFLOW: return "MAP_E_OVERFLOW";
    case MAP_E_TIMEOUT: return "MAP_E_TIMEOUT";
    case MAP_E_STATE: return "MAP_E_STATE";
    case MAP_E_INTERNAL: return "MAP_E_INTERNAL";
  }
  return "MAP_E_UNKNOWN";
}

map_status map_create(const int64_t* xadj, const int32_t* adjncy, const int32_t* adjwgt, const int32_t* vwgt,
                      int32_t n, const int32_t* hier, const int32_t* dist, int32_t levels, double eps,
                      const map_config* cfg, void* stream, int32_t inputs_on_device, map_ctx** out) {
  if (!out) return MAP_E_INVALID;
  *out = nullptr;
  map_ctx* ctx = new (std::nothrow) map_ctx();
  if (!ctx) return MAP_E_OOM;
  map_status st = guarded(ctx, [&](Ctx& c) {
    if (n < 1) throw ApiError(MAP_E_INVALID, "n must be >= 1");
    if (!xadj || !hier || !dist) throw ApiError(MAP_E_INVALID, "xadj, hier and dist are required");
    if (!(eps >= 0.0 && eps < 1.0)) throw ApiError(MAP_E_INVALID, "eps must be in [0, 1)");
    if (cfg) c.cfg = *cfg;
    else map_config_default(&c.cfg);
    if (c.cfg.patience < 1 || c.cfg.weak_max < 0 || c.cfg.phi_den < 1 || c.cfg.phi_num < 0 ||
        c.cfg.coarsest_factor < 1 || c.cfg.cluster_iters < 0 || c.cfg.cluster_cap_div < 1 || c.cfg.max_levels < 1 ||
        c.cfg.max_levels > 64 || c.cfg.stall_den < 1)
      throw ApiError(MAP_E_INVALID, "map_config field out of range");
    if (c.cfg.launch_mode < 0 || c.cfg.launch_mode > 1) throw ApiError(MAP_E_INVALID, "launch_mode must be 0 or 1");
    c.use_graphs = c.cfg.launch_mode == 0;
    if (c.cfg.engine_max_n < -1 || c.cfg.grid_engine_max_n < -1)
      throw ApiError(MAP_E_INVALID, "engine_max_n and grid_engine_max_n must be >= -1");
    if (c.cfg.coarsener < 0 || c.cfg.coarsener > 1 || c.cfg.match_rounds < 0)
      throw ApiError(MAP_E_INVALID, "coarsener must be 0 or 1 and match_rounds >= 0");
    if (c.cfg.initial < 0 || c.cfg.initial > 1) throw ApiError(MAP_E_INVALID, "initial must be 0 or 1");
    if (c.cfg.lp_relax_num < 0 || c.cfg.lp_relax_den < 1)
      throw ApiError(MAP_E_INVALID, "lp_relax_num must be >= 0 and lp_relax_den >= 1");
    if (c.cfg.reb_objective < 0 || c.cfg.reb_objective > 1)
      throw ApiError(MAP_E_INVALID, "reb_objective must be 0 or 1");
    if (c.cfg.mid_deg != 0 && (c.cfg.mid_deg <= kLowDeg || c.cfg.mid_deg > kMidDeg))
      throw ApiError(MAP_E_INVALID, "mid_deg must be 0 (autotuned) or in 33..255");
    if (c.cfg.split_deg < 0) throw ApiError(MAP_E_INVALID, "split_deg must be 0 (autotuned) or positive");
    c.st = (cudaStream_t)stream;
    GM_CUDA(cudaGetDevice(&c.dev));
    sort_init();
    GM_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.dev));
    if (!c.cfg.alloc) keep_pool_memory(c.dev);
    c.mem.st = c.st;
    c.mem.afn = c.cfg.alloc;
    c.mem.ffn = c.cfg.free;
    c.mem.user = c.cfg.alloc_user;
    build_topology(c, hier, dist, levels);
    c.eps = eps;
    c.lv.reserve(66);
    int64_t m = 0;
    if (inputs_on_device) {
      GM_CUDA(cudaMemcpyAsync(&m, xadj + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
      sync(c);
    } else {
      m = xadj[n];
      if (xadj[0] != 0) throw ApiError(MAP_E_INVALID, "xadj[0] must be 0");
    }
    if (m < 0 || m >= (1LL << 40)) throw ApiError(MAP_E_INVALID, "xadj[n] out of range");
    if (m > 0 && !adjncy) throw ApiError(MAP_E_INVALID, "adjncy is required when the graph has edges");
    c.n0 = n;
    c.m0 = m;
    Level L;
    L.n = n;
    L.m = m;
    L.xadj = c.mem.make<int64_t>((size_t)n + 1);
    L.adj = c.mem.make<int32_t>((size_t)std::max<int64_t>(1, m));
    L.adjw = c.mem.make<int32_t>((size_t)std::max<int64_t>(1, m));
    L.vw = c.mem.make<int32_t>((size_t)n);
    L.pi = c.mem.make<int32_t>((size_t)n);
    const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    GM_CUDA(cudaMemcpyAsync(L.xadj, xadj, ((size_t)n + 1) * sizeof(int64_t), kind, c.st));
    if (m > 0) GM_CUDA(cudaMemcpyAsync(L.adj, adjncy, (size_t)m * sizeof(int32_t), kind, c.st));
    if (adjwgt) {
      if (m > 0) GM_CUDA(cudaMemcpyAsync(L.adjw, adjwgt, (size_t)m * sizeof(int32_t), kind, c.st));
    } else {
      std::vector<int32_t> ones((size_t)std::max<int64_t>(1, m), 1);
      GM_CUDA(cudaMemcpyAsync(L.adjw, ones.data(), ones.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.st));
      sync(c);
    }
    if (vwgt) {
      GM_CUDA(cudaMemcpyAsync(L.vw, vwgt, (size_t)n * sizeof(int32_t), kind, c.st));
    } else {
      std::vector<int32_t> ones((size_t)n, 1);
      GM_CUDA(cudaMemcpyAsync(L.vw, ones.data(), ones.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.st));
      sync(c);
    }
    GM_CUDA(cudaMemsetAsync(L.pi, 0, (size_t)n * sizeof(int32_t), c.st));
    c.lv.push_back(L);
    c.d_code_of_pe = c.mem.make<int32_t>((size_t)c.k);
    c.d_pe_of_code = c.mem.make<int32_t>((size_t)c.topo.kc);
    const size_t tk = (size_t)c.k * sizeof(int32_t), tc = (size_t)c.topo.kc * sizeof(int32_t);
    const int32_t* src_k = c.code_of_pe.data();
    const int32_t* src_c = c.pe_of_code.data();
    if (tk + tc <= kPinnedBlock) {  // small tables travel from pinned memory (no shared staging buffer)
      c.h_tables = pinned_get(tk + tc);
      std::memcpy(c.h_tables, src_k, tk);
      std::memcpy(static_cast<char*>(c.h_tables) + tk, src_c, tc);
      src_k = static_cast<const int32_t*>(c.h_tables);
      src_c = reinterpret_cast<const int32_t*>(static_cast<const char*>(c.h_tables) + tk);
    }
    GM_CUDA(cudaMemcpyAsync(c.d_code_of_pe, src_k, tk, cudaMemcpyHostToDevice, c.st));
    GM_CUDA(cudaMemcpyAsync(c.d_pe_of_code, src_c, tc, cudaMemcpyHostToDevice, c.st));
    c.errword = reinterpret_cast<uint32_t*>(c.mem.make<int64_t>(1));
    alloc_sort(c);
    refine_alloc(c);
    coarsen_alloc(c);
    validate_graph(c);
    classify_degrees(c, 0);
    c.lmax = lmax_of(c.cV, c.k, eps);
    sync(c);
  });
  if (st != MAP_OK) {
    // keep the context alive so that map_last_error can report; free memory now
    try {
      ctx->c.mem.release_all();
      pinned_put(ctx->c.h_state);
      ctx->c.h_state = nullptr;
      pinned_put(ctx->c.h_cstate);
      ctx->c.h_cstate = nullptr;
      pinned_put(ctx->c.h_small);
      ctx->c.h_small = nullptr;
      pinned_put(ctx->c.h_tables);
      ctx->c.h_tables = nullptr;
      cudaStreamSynchronize(ctx->c.st);
      for (auto& cs : ctx->c.cap.s)
        if (cs) cudaStreamDestroy(cs);
    } catch (...) {
    }
    last_create_error() = ctx->c.err;
    delete ctx;
    *out = nullptr;
    return st;
  }
  *out = ctx;
  return MAP_OK;
}

void map_destroy(map_ctx* ctx) {
  if (!ctx) return;
  try {
    cudaStreamSynchronize(ctx->c.st);
    ctx->c.mem.release_all();
    cudaStreamSynchronize(ctx->c.st);
    pinned_put(ctx->c.h_state);
    pinned_put(ctx->c.h_cstate);
    pinned_put(ctx->c.h_small);
    pinned_put(ctx->c.h_eng_job);
    pinned_put(ctx->c.h_tables);
    for (cudaEvent_t e : ctx->c.ev_pool) cudaEventDestroy(e);
    for (auto& L : ctx->c.lv) {
      drop_graph(L);
      if (L.cgexec) cudaGraphExecDestroy(L.cgexec);
    }
    for (auto& cs : ctx->c.cap.s)
      if (cs) cudaStreamDestroy(cs);
  } catch (...) {
  }
  delete ctx;
}

const char* map_last_error(const map_ctx* ctx) { return ctx ? ctx->c.err.c_str() : last_create_error().c_str(); }

map_status map_sync(map_ctx* ctx) {
  return guarded(ctx, [&](Ctx& c) { sync(c); });
}

map_status map_info(const map_ctx* cctx, int32_t* out_k, int64_t* out_lmax, int64_t* out_total_weight) {
  if (!cctx) return MAP_E_INVALID;
  if (out_k) *out_k = cctx->c.k;
  if (out_lmax) *out_lmax = cctx->c.lmax;
  if (out_total_weight) *out_total_weight = cctx->c.cV;
  return MAP_OK;
}

map_status map_set_mapping(map_ctx* ctx, int32_t level, const int32_t* pi) {
  return guarded(ctx, [&](Ctx& c) {
    Level& L = level_at(c, level);
    if (!pi) throw ApiError(MAP_E_INVALID, "pi is NULL");
    std::vector<int32_t> codes((size_t)L.n);
    for (int32_t v = 0; v < L.n; v++) {
      if (pi[v] < 0 || pi[v] >= c.k) throw ApiError(MAP_E_INVALID, "mapping entry out of [0, k)");
      codes[(size_t)v] = c.code_of_pe[(size_t)pi[v]];
    }
    GM_CUDA(cudaMemcpyAsync(L.pi, codes.data(), codes.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.st));
    sync(c);
  });
}

map_status map_get_mapping(map_ctx* ctx, int32_t level, int32_t* pi) {
  return guarded(ctx, [&](Ctx& c) {
    Level& L = level_at(c, level);
    if (!pi) throw ApiError(MAP_E_INVALID, "pi is NULL");
    GM_CUDA(cudaMemcpyAsync(pi, L.pi, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    sync(c);
    for (int32_t v = 0; v < L.n; v++) pi[v] = c.pe_of_code[(size_t)pi[v]];
  });
}

map_status map_objective(map_ctx* ctx, int32_t level, int64_t* out_J, int64_t* out_max_block_weight) {
  return guarded(ctx, [&](Ctx& c) {
    level_at(c, level);
    objective(c, level, out_J, out_max_block_weight);
  });
}

map_status map_block_weights(map_ctx* ctx, int32_t level, int64_t* out_W) {
  return guarded(ctx, [&](Ctx& c) {
    level_at(c, level);
    if (!out_W) throw ApiError(MAP_E_INVALID, "out_W is NULL");
    compute_block_weights(c, level);
    std::vector<int64_t> W((size_t)c.topo.kc);
    GM_CUDA(cudaMemcpyAsync(W.data(), c.W, W.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
    sync(c);
    for (int32_t p = 0; p < c.k; p++) out_W[p] = W[(size_t)c.code_of_pe[(size_t)p]];
  });
}

map_status map_lp_step(map_ctx* ctx, int32_t level, int32_t* out_moved) {
  return guarded(ctx, [&](Ctx& c) {
    level_at(c, level);
    const int32_t mv = lp_step(c, level);
    if (out_moved) *out_moved = mv;
  });
}

map_status map_get_lp_state(map_ctx* ctx, int32_t level, int32_t* pi_prime, int64_t* gain, uint8_t* in_x,
                            uint8_t* moved) {
  return guarded(ctx, [&](Ctx& c) {
    Level& L = level_at(c, level);
    const size_t n = (size_t)L.n;
    if (pi_prime) GM_CUDA(cudaMemcpyAsync(pi_prime, c.pp, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    if (gain) GM_CUDA(cudaMemcpyAsync(gain, c.gain, n * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
    if (in_x) GM_CUDA(cudaMemcpyAsync(in_x, c.inx, n, cudaMemcpyDeviceToHost, c.st));
    if (moved) GM_CUDA(cudaMemcpyAsync(moved, c.lock, n, cudaMemcpyDeviceToHost, c.st));
    sync(c);
    if (pi_prime)
      for (size_t v = 0; v < n; v++) pi_prime[v] = c.pe_of_code[(size_t)pi_prime[v]];
  });
}

map_status map_set_lock(map_ctx* ctx, int32_t level, const uint8_t* lock) {
  return guarded(ctx, [&](Ctx& c) {
    Level& L = level_at(c, level);
    if (!lock) throw ApiError(MAP_E_INVALID, "lock is NULL");
    std::vector<uint8_t> h(lock, lock + L.n);
    for (auto& x : h) x = x ? 1 : 0;
    GM_CUDA(cudaMemcpyAsync(c.lock, h.data(), h.size(), cudaMemcpyHostToDevice, c.st));
    sync(c);
  });
}

map_status map_rebalance_step(map_ctx* ctx, int32_t level, int32_t strong, int32_t t, int32_t* out_moved) {
  return guarded(ctx, [&](Ctx& c) {
    level_at(c, level);
    const int32_t mv = rebalance_step(c, level, strong != 0, t);
    if (out_moved) *out_moved = mv;
  });
}

map_status map_refine(map_ctx* ctx, int32_t level, int32_t rounds, int64_t* out_J, int64_t* out_max_block_weight,
                      int32_t* out_iters) {
  return guarded(ctx, [&](Ctx& c) {
    level_at(c, level);
    refine(c, level, rounds, out_J, out_max_block_weight, out_iters);
    sync(c);
  });
}

map_status map_get_refine_trace(map_ctx* ctx, int32_t cap, int32_t* kind, int64_t* J, int64_t* max_block_weight,
                                int32_t* out_count) {
  return guarded(ctx, [&](Ctx& c) {
    const int32_t cnt = std::min(std::min(cap, c.trace_cap), c.last_iters);
    if (cnt > 0) {
      if (kind) GM_CUDA(cudaMemcpyAsync(kind, c.trace_kind, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
      if (J) GM_CUDA(cudaMemcpyAsync(J, c.trace_J, cnt * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
      if (max_block_weight)
        GM_CUDA(cudaMemcpyAsync(max_block_weight, c.trace_maxw, cnt * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
      sync(c);
    }
    if (out_count) *out_count = c.last_iters;
  });
}

map_status map_coarsen(map_ctx* ctx, int32_t* out_levels) {
  return guarded(ctx, [&](Ctx& c) {
    const double t0 = now_ms();
    const int32_t l = coarsen(c);
    sync(c);
    c.ms_coarsen = now_ms() - t0;
    if (out_levels) *out_levels = l;
  });
}

map_status map_level_info(map_ctx* ctx, int32_t level, int32_t* out_n, int64_t* out_m_dir) {
  return guarded(ctx, [&](Ctx& c) {
    Level& L = level_at(c, level);
    if (out_n) *out_n = L.n;
    if (out_m_dir) *out_m_dir = L.m;
  });
}

map_status map_get_level_graph(map_ctx* ctx, int32_t level, int64_t* xadj, int32_t* adjncy, int32_t* adjwgt,
                               int32_t* vwgt, int32_t* M) {
  return guarded(ctx, [&](Ctx& c) {
    Level& L = level_at(c, level);
    if (xadj) GM_CUDA(cudaMemcpyAsync(xadj, L.xadj, ((size_t)L.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c.st));
    if (adjncy && L.m) GM_CUDA(cudaMemcpyAsync(adjncy, L.adj, (size_t)L.m * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    if (adjwgt && L.m) GM_CUDA(cudaMemcpyAsync(adjwgt, L.adjw, (size_t)L.m * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    if (vwgt) GM_CUDA(cudaMemcpyAsync(vwgt, L.vw, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    if (M) {
      if (!L.M) throw ApiError(MAP_E_STATE, "level has no coarser level");
      GM_CUDA(cudaMemcpyAsync(M, L.M, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    }
    sync(c);
  });
}

map_status map_initial(map_ctx* ctx) {
  return guarded(ctx, [&](Ctx& c) {
    const double t0 = now_ms();
    initial_map(c);
    sync(c);
    c.ms_initial = now_ms() - t0;
  });
}

map_status map_project(map_ctx* ctx, int32_t level) {
  return guarded(ctx, [&](Ctx& c) {
    if (level < 0 || level + 1 >= (int32_t)c.lv.size() || !c.lv[(size_t)level].M)
      throw ApiError(MAP_E_STATE, "level has no coarser level to project from");
    project(c, level);
  });
}

map_status map_run(map_ctx* ctx, int32_t* out_pi, int64_t* out_J) {
  return guarded(ctx, [&](Ctx& c) {
    double t0 = now_ms();
    coarsen(c);
    sync(c);
    c.ms_coarsen = now_ms() - t0;
    t0 = now_ms();
    initial_map(c);
    c.ms_initial = now_ms() - t0;
    c.ms_refine = 0;
    c.ms_project = 0;
    const int top = (int)c.lv.size() - 1;
    int64_t J = 0, mw = 0;
    for (int l = top; l >= 0; l--) {
      if (l < top) {
        t0 = now_ms();
        project(c, l);
        c.ms_project += now_ms() - t0;
      }
      t0 = now_ms();
      int32_t it = 0;
      refine(c, l, -1, &J, &mw, &it);
      const double dt = now_ms() - t0;
      c.ms_refine += dt;
      if (l <= 64) {
        c.iters[l] = it;
        c.Jlev[l] = J;
        c.ms_level[l] = dt;
        // the kinds of the level's iterations (the trace holds the first trace_cap)
        const int32_t cnt = std::min(it, c.trace_cap);
        c.kinds[l][0] = c.kinds[l][1] = c.kinds[l][2] = 0;
        if (cnt > 0) {
          std::vector<int32_t> tk((size_t)cnt);
          GM_CUDA(cudaMemcpyAsync(tk.data(), c.trace_kind, (size_t)cnt * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  c.st));
          sync(c);
          for (int32_t k : tk)
            if (k >= KIND_LP && k <= KIND_STRONG) c.kinds[l][k]++;
        }
      }
    }
    if (out_pi) {
      Level& L = c.lv[0];
      GM_CUDA(cudaMemcpyAsync(out_pi, L.pi, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
      sync(c);
      for (int32_t v = 0; v < L.n; v++) out_pi[v] = c.pe_of_code[(size_t)out_pi[v]];
    }
    if (out_J) *out_J = J;
  });
}

map_status map_run_hm(map_ctx* ctx, int32_t workers, int32_t* out_pi, int64_t* out_J) {
  return guarded(ctx, [&](Ctx& c) {
    if (workers < 0) throw ApiError(MAP_E_INVALID, "workers must be >= 0");
    hm_run(c, 0, workers ? workers : 8, &c.hm);
    int64_t J = 0, mw = 0;
    objective(c, 0, &J, &mw);
    if (out_pi) {
      Level& L = c.lv[0];
      GM_CUDA(cudaMemcpyAsync(out_pi, L.pi, (size_t)L.n * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
      sync(c);
      for (int32_t v = 0; v < L.n; v++) out_pi[v] = c.pe_of_code[(size_t)out_pi[v]];
    }
    if (out_J) *out_J = J;
  });
}

map_status map_hm_stats(map_ctx* ctx, int32_t which, map_hm_stats_t* out) {
  return guarded(ctx, [&](Ctx& c) {
    if (!out) throw ApiError(MAP_E_INVALID, "out is NULL");
    if (which < 0 || which > 1) throw ApiError(MAP_E_INVALID, "which must be 0 or 1");
    const HmStats& h = which == 0 ? c.hm : c.hm_init;
    std::memset(out, 0, sizeof(*out));
    out->levels = h.levels;
    out->workers = h.workers;
    for (int i = 0; i < 16; i++) {
      out->calls[i] = h.calls[i];
      out->first_eps[i] = h.first_eps[i];
      out->ms_level[i] = h.ms_level[i];
    }
    out->ms_partition = h.ms_partition;
    out->ms_build = h.ms_build;
    out->ms_total = h.ms_total;
    out->ms_create = h.ms_create;
    out->ms_run = h.ms_run;
    out->ms_destroy = h.ms_destroy;
  });
}

map_status map_stats(map_ctx* ctx, map_stats_t* out) {
  return guarded(ctx, [&](Ctx& c) {
    if (!out) throw ApiError(MAP_E_INVALID, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->levels = (int32_t)c.lv.size();
    for (size_t l = 0; l < c.lv.size() && l < 65; l++) {
      out->n[l] = c.lv[l].n;
      out->m_dir[l] = c.lv[l].m;
      out->J[l] = c.Jlev[l];
      out->iters[l] = c.iters[l];
      out->ms_refine_level[l] = c.ms_level[l];
      out->mid_deg[l] = c.lv[l].mid_deg;
      out->split_deg[l] = (int32_t)std::min<int64_t>(c.lv[l].hub_split_deg, INT32_MAX);
      out->tuned[l] = c.lv[l].tuned;
      out->lp_iters[l] = c.kinds[l][KIND_LP];
      out->weak_iters[l] = c.kinds[l][KIND_WEAK];
      out->strong_iters[l] = c.kinds[l][KIND_STRONG];
    }
    out->ms_tune = c.ms_tune;
    out->ms_coarsen = c.ms_coarsen;
    out->ms_initial = c.ms_initial;
    out->ms_refine = c.ms_refine;
    out->ms_project = c.ms_project;
    out->device_bytes = (int64_t)c.mem.total;
    out->device_bytes_peak = (int64_t)c.mem.peak;
  });
}

map_status map_profile_enable(map_ctx* ctx, int32_t enable) {
  return guarded(ctx, [&](Ctx& c) {
    sync(c);
    c.prof = enable != 0;
    c.prof_recs.clear();
    c.ev_used = 0;
  });
}

map_status map_profile_read(map_ctx* ctx, int32_t which, int32_t level, int64_t* launches, double* total_ms,
                            int64_t* bytes) {
  return guarded(ctx, [&](Ctx& c) {
    if (which < 0 || which >= PK_COUNT) throw ApiError(MAP_E_INVALID, "unknown kernel class");
    sync(c);
    int64_t cnt = 0, by = 0;
    double ms = 0;
    std::vector<ProfRec> keep;
    for (const ProfRec& r : c.prof_recs) {
      if (r.kind != which || (level >= 0 && r.level != level)) {
        keep.push_back(r);
        continue;
      }
      float t = 0;
      GM_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      ms += t;
      by += r.bytes;
      cnt++;
    }
    c.prof_recs.swap(keep);
    if (c.prof_recs.empty()) c.ev_used = 0;
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    if (bytes) *bytes = by;
  });
}

long long map_launch_count(void) { return gm::launch_count(); }

map_status map_selftest_barrier_timeout(void* stream) {
  last_create_error().clear();
  try {
    if (!barrier_selftest((cudaStream_t)stream)) {
      last_create_error() = "the grid barrier was released or did not report the expired wait";
      return MAP_E_INTERNAL;
    }
    last_create_error() = "a grid barrier wait expired (expected by this self-test)";
    return MAP_E_TIMEOUT;
  } catch (const CudaError& e) {
    last_create_error() = e.what();
    return MAP_E_CUDA;
  } catch (const std::exception& e) {
    last_create_error() = e.what();
    return MAP_E_INTERNAL;
  }
}

}  // extern "C"
