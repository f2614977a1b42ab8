// Batched refinement: many contexts (graphs of uneven size, each with its own
// hierarchy and distances) refined in one persistent launch of the fused
// Alg. 6 engine, captured once in a CUDA graph and replayed.
//
// Every job is processed from start to end by one thread-block cluster: the
// clusters of the persistent grid take jobs from a device counter, largest
// job first (longest-processing-time order), so small jobs fill the gaps
// left by large ones.  Each job keeps its own context's buffers, hence the
// result of a job does not depend on the schedule (cluster size, staging
// capacity, order, which cluster took it): it equals map_refine on the same
// context.  The schedule is chosen by timing the candidates on the batch
// itself (with the mappings restored before every trial), and the choice is
// cached per batch signature for later batches of the same shape.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

namespace gm {
namespace {

struct JobResult {
  int64_t J;
  int64_t maxw;
  int64_t iters;
  int64_t capped;
};

__global__ void k_batch_collect(RefineState* const* __restrict__ states, int32_t njobs, JobResult* out) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < njobs; i += gridDim.x * blockDim.x) {
    const RefineState* s = states[i];
    out[i] = JobResult{s->best_J, s->best_maxw, s->t, s->capped};
  }
}

struct Schedule {
  int C = 0;    // CTAs per cluster (one cluster per job at a time)
  int te = 0;   // staged CSR entries per warp tile
  int ncl = 0;  // clusters of the persistent grid
  double ms = 0.0;
};

double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

using Signature = std::tuple<int, int32_t, int32_t, int64_t, int64_t, int32_t, int32_t>;
std::mutex g_tune_mutex;
std::map<Signature, Schedule> g_tune_cache;

}  // namespace
}  // namespace gm

using namespace gm;

struct map_batch {
  std::vector<map_ctx*> jobs;
  map_batch_opts opts{};
  int dev = 0;
  cudaStream_t st = nullptr;       // caller's stream
  cudaStream_t cap = nullptr;      // private stream for capture and tuning
  std::vector<int32_t> order;      // job indices, largest first
  std::vector<uint64_t> gens;      // each job's level generation when the batch was built
  void* d_jobs = nullptr;          // engine job descriptors in `order`
  RefineState** d_states = nullptr;
  JobResult* d_res = nullptr;
  JobResult* h_res = nullptr;
  unsigned int* d_queue = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long graph_kernels = 0;     // kernel launches per replay
  cudaEvent_t ev_in = nullptr, ev_done = nullptr;
  Schedule sched;
  bool tuned = false;
  bool var = false;                // some job uses the refinement variants (512-entry tiles only)
  double tune_ms = 0.0;
  int32_t max_n = 0;
  int64_t sum_n = 0, sum_m = 0;
  std::string err;
};

namespace {

void release(map_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_jobs) cudaFree(b->d_jobs);
  if (b->d_states) cudaFree(b->d_states);
  if (b->d_res) cudaFree(b->d_res);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->h_res) cudaFreeHost(b->h_res);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaGetLastError();
}

template <class F>
map_status batch_guard(map_batch* b, F&& f) {
  if (!b) return MAP_E_INVALID;
  try {
    b->err.clear();
    f(*b);
    return MAP_OK;
  } catch (const ApiError& e) {
    b->err = e.what();
    return e.status;
  } catch (const CudaError& e) {
    b->err = e.what();
    return e.code == cudaErrorMemoryAllocation ? MAP_E_OOM : MAP_E_CUDA;
  } catch (const std::bad_alloc&) {
    b->err = "host allocation failed";
    return MAP_E_OOM;
  } catch (const std::exception& e) {
    b->err = e.what();
    return MAP_E_INTERNAL;
  }
}

// The jobs' pending work (on their own streams) before stream `s`.
void wait_for_jobs(map_batch& b, cudaStream_t s) {
  for (map_ctx* j : b.jobs) {
    GM_CUDA(cudaEventRecord(b.ev_in, j->c.st));
    GM_CUDA(cudaStreamWaitEvent(s, b.ev_in, 0));
  }
}

// Later work of every job (on its stream) after the batch on stream `s`.
void jobs_wait_for(map_batch& b, cudaStream_t s) {
  GM_CUDA(cudaEventRecord(b.ev_done, s));
  for (map_ctx* j : b.jobs) GM_CUDA(cudaStreamWaitEvent(j->c.st, b.ev_done, 0));
}

void enqueue(map_batch& b, cudaStream_t s, const Schedule& sc) {
  GM_CUDA(cudaMemsetAsync(b.d_queue, 0, sizeof(unsigned int), s));
  engine_launch(s, b.d_jobs, (int)b.jobs.size(), b.d_queue, sc.C, sc.te, sc.ncl, b.var);
  k_batch_collect<<<1, 256, 0, s>>>(b.d_states, (int32_t)b.jobs.size(), b.d_res); count_launch();
}

Schedule make_schedule(map_batch& b, int C, int te) {
  Schedule sc;
  const int resident = engine_max_clusters(C, te);
  if (resident < 1) return sc;
  sc.C = C;
  sc.te = te;
  sc.ncl = std::min<int>(resident, (int)b.jobs.size());
  return sc;
}

// Automatic schedule without timing: enough CTAs per job that the largest
// job does not dominate, at least as many clusters as fit.
Schedule default_schedule(map_batch& b) {
  int C = 1;
  while (C < 16 && (int64_t)C * 4096 < b.max_n) C *= 2;
  Schedule sc = make_schedule(b, C, b.opts.tile_entries ? b.opts.tile_entries : 512);
  while (sc.C == 0 && C > 1) {
    C /= 2;
    sc = make_schedule(b, C, b.opts.tile_entries ? b.opts.tile_entries : 512);
  }
  if (sc.C == 0) throw ApiError(MAP_E_CUDA, "the refinement engine cannot be launched on this device");
  return sc;
}

// Times every candidate schedule once on the batch (mappings restored before
// each trial and at the end) and returns the fastest.
Schedule autotune(map_batch& b) {
  const size_t nj = b.jobs.size();
  std::vector<int32_t*> saved(nj, nullptr);
  std::vector<size_t> bytes(nj);
  Schedule best;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    for (int32_t* p : saved)
      if (p) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  try {
    GM_CUDA(cudaEventCreate(&e0));
    GM_CUDA(cudaEventCreate(&e1));
    for (size_t i = 0; i < nj; i++) {
      const Level& L = b.jobs[i]->c.lv[b.opts.level];
      bytes[i] = (size_t)L.n * sizeof(int32_t);
      GM_CUDA(cudaMalloc(&saved[i], bytes[i]));
      GM_CUDA(cudaMemcpyAsync(saved[i], L.pi, bytes[i], cudaMemcpyDeviceToDevice, b.cap));
    }
    auto restore = [&]() {
      for (size_t i = 0; i < nj; i++)
        GM_CUDA(cudaMemcpyAsync(b.jobs[i]->c.lv[b.opts.level].pi, saved[i], bytes[i], cudaMemcpyDeviceToDevice,
                                b.cap));
    };
    std::vector<Schedule> cand;
    for (int te : {512, 256})
      for (int C : {1, 2, 4, 8, 16}) {
        if (b.var && te != 512) continue;
        const Schedule sc = make_schedule(b, C, te);
        if (sc.C) cand.push_back(sc);
      }
    if (cand.empty()) throw ApiError(MAP_E_CUDA, "the refinement engine cannot be launched on this device");
    enqueue(b, b.cap, cand[0]);  // warm-up (first launch of the module)
    for (Schedule& sc : cand) {
      restore();
      GM_CUDA(cudaEventRecord(e0, b.cap));
      enqueue(b, b.cap, sc);
      GM_CUDA(cudaEventRecord(e1, b.cap));
      GM_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      GM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      sc.ms = ms;
      if (best.C == 0 || sc.ms < best.ms) best = sc;
    }
    restore();
    GM_CUDA(cudaStreamSynchronize(b.cap));
  } catch (...) {
    cudaStreamSynchronize(b.cap);
    cleanup();
    throw;
  }
  cleanup();
  return best;
}

void capture(map_batch& b) {
  GM_CUDA(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal));
  long long* prev = set_capture_counter(&b.graph_kernels);
  try {
    enqueue(b, b.cap, b.sched);
    set_capture_counter(prev);
  } catch (...) {
    set_capture_counter(prev);
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(b.cap, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  GM_CUDA(cudaStreamEndCapture(b.cap, &b.graph));
  GM_CUDA(cudaGraphInstantiate(&b.exec, b.graph, 0));
}

}  // namespace

extern "C" {

void map_batch_opts_default(map_batch_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->level = 0;
  o->rounds = 10;
  o->autotune = 1;
}

map_status map_batch_create(map_ctx* const* jobs, int32_t njobs, const map_batch_opts* opts, void* stream,
                            map_batch** out) {
  if (!out) return MAP_E_INVALID;
  *out = nullptr;
  map_batch* b = new (std::nothrow) map_batch();
  if (!b) return MAP_E_OOM;
  const map_status st = batch_guard(b, [&](map_batch& B) {
    if (!jobs || njobs < 1) throw ApiError(MAP_E_INVALID, "jobs must hold njobs >= 1 contexts");
    if (opts) B.opts = *opts;
    else map_batch_opts_default(&B.opts);
    if (B.opts.rounds == 0 || B.opts.rounds < -1 || B.opts.rounds > kMaxRefineIters)
      throw ApiError(MAP_E_INVALID, "rounds must be -1 (Alg. 6 termination) or in [1, 2^20)");
    if (B.opts.tile_entries != 0 && B.opts.tile_entries != 256 && B.opts.tile_entries != 512)
      throw ApiError(MAP_E_INVALID, "tile_entries must be 0, 256 or 512");
    if (B.opts.cluster != 0 && B.opts.cluster != 1 && B.opts.cluster != 2 && B.opts.cluster != 4 &&
        B.opts.cluster != 8 && B.opts.cluster != 16)
      throw ApiError(MAP_E_INVALID, "cluster must be 0, 1, 2, 4, 8 or 16");
    GM_CUDA(cudaGetDevice(&B.dev));
    B.st = (cudaStream_t)stream;
    B.jobs.assign(jobs, jobs + njobs);
    for (int32_t i = 0; i < njobs; i++) {
      map_ctx* j = B.jobs[i];
      if (!j) throw ApiError(MAP_E_INVALID, "job " + std::to_string(i) + " is NULL");
      for (int32_t k = 0; k < i; k++)
        if (B.jobs[k] == j) throw ApiError(MAP_E_INVALID, "job " + std::to_string(i) + " repeats job " + std::to_string(k));
      if (j->c.dev != B.dev) throw ApiError(MAP_E_INVALID, "job " + std::to_string(i) + " lives on another device");
      if (B.opts.level < 0 || B.opts.level >= (int)j->c.lv.size() || !j->c.lv[B.opts.level].pi)
        throw ApiError(MAP_E_STATE, "job " + std::to_string(i) + " has no level " + std::to_string(B.opts.level));
      B.var = B.var || uses_variants(j->c.cfg);
    }
    if (B.var && B.opts.tile_entries == 256)
      throw ApiError(MAP_E_INVALID, "jobs with the refinement variants need tile_entries 0 or 512");
    GM_CUDA(cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking));
    GM_CUDA(cudaEventCreateWithFlags(&B.ev_in, cudaEventDisableTiming));
    GM_CUDA(cudaEventCreateWithFlags(&B.ev_done, cudaEventDisableTiming));
    // largest job first
    B.order.resize(njobs);
    for (int32_t i = 0; i < njobs; i++) B.order[i] = i;
    auto work = [&](int32_t i) {
      const Level& L = B.jobs[i]->c.lv[B.opts.level];
      return (int64_t)L.n + L.m;
    };
    std::stable_sort(B.order.begin(), B.order.end(), [&](int32_t x, int32_t y) { return work(x) > work(y); });
    const size_t jb = engine_job_bytes();
    std::vector<unsigned char> hj(jb * njobs);
    std::vector<RefineState*> hs(njobs);
    for (int32_t r = 0; r < njobs; r++) {
      const int32_t i = B.order[r];
      Ctx& c = B.jobs[i]->c;
      if (!engine_job_write(c, B.opts.level, B.opts.rounds, hj.data() + jb * r))
        throw ApiError(MAP_E_INVALID, "job " + std::to_string(i) +
                                          ": the level has a row of degree > 128 and a PE code space whose "
                                          "connectivity table does not fit in shared memory; refine it with "
                                          "map_refine");
      const Level& L = c.lv[B.opts.level];
      B.max_n = std::max(B.max_n, L.n);
      B.sum_n += L.n;
      B.sum_m += L.m;
    }
    for (int32_t i = 0; i < njobs; i++) hs[i] = B.jobs[i]->c.state;
    B.gens.resize(njobs);
    for (int32_t i = 0; i < njobs; i++) B.gens[i] = B.jobs[i]->c.level_gen;
    GM_CUDA(cudaMalloc(&B.d_jobs, jb * njobs));
    GM_CUDA(cudaMalloc(&B.d_states, sizeof(RefineState*) * njobs));
    GM_CUDA(cudaMalloc(&B.d_res, sizeof(JobResult) * njobs));
    GM_CUDA(cudaMalloc(&B.d_queue, sizeof(unsigned int)));
    GM_CUDA(cudaMallocHost(&B.h_res, sizeof(JobResult) * njobs));
    GM_CUDA(cudaMemcpyAsync(B.d_jobs, hj.data(), jb * njobs, cudaMemcpyHostToDevice, B.cap));
    GM_CUDA(cudaMemcpyAsync(B.d_states, hs.data(), sizeof(RefineState*) * njobs, cudaMemcpyHostToDevice, B.cap));
    GM_CUDA(cudaStreamSynchronize(B.cap));
  });
  if (st != MAP_OK) {
    last_create_error() = b->err;
    release(b);
    delete b;
    return st;
  }
  *out = b;
  return MAP_OK;
}

map_status map_batch_launch(map_batch* b) {
  return batch_guard(b, [&](map_batch& B) {
    GM_CUDA(cudaSetDevice(B.dev));
    // the job descriptors and the captured graph hold pointers into the
    // jobs' level buffers, which a coarsening (map_coarsen, map_run) may move
    for (size_t i = 0; i < B.jobs.size(); i++)
      if (B.jobs[i]->c.level_gen != B.gens[i])
        throw ApiError(MAP_E_STATE, "job " + std::to_string(i) +
                                        " was coarsened after the batch was built (map_coarsen or map_run); "
                                        "destroy the batch and build a new one");
    if (!B.tuned) {
      // the jobs' mappings must be in place before tuning or capture
      wait_for_jobs(B, B.cap);
      if (B.opts.autotune) {
        const Signature key{B.dev, (int32_t)B.jobs.size(), B.max_n, B.sum_n, B.sum_m, B.opts.rounds, B.opts.level};
        bool hit = false;
        {
          std::lock_guard<std::mutex> lock(g_tune_mutex);
          auto it = g_tune_cache.find(key);
          if (it != g_tune_cache.end()) {
            B.sched = it->second;
            hit = true;
          }
        }
        if (!hit) {
          GM_CUDA(cudaStreamSynchronize(B.cap));
          const double t0 = wall_ms();
          B.sched = autotune(B);
          B.tune_ms = wall_ms() - t0;
          std::lock_guard<std::mutex> lock(g_tune_mutex);
          g_tune_cache[key] = B.sched;
        }
      } else if (B.opts.cluster) {
        B.sched = make_schedule(B, B.opts.cluster, B.opts.tile_entries ? B.opts.tile_entries : 512);
        if (!B.sched.C) throw ApiError(MAP_E_INVALID, "the requested cluster size cannot be launched on this device");
      } else {
        B.sched = default_schedule(B);
      }
      capture(B);
      B.tuned = true;
      GM_CUDA(cudaStreamSynchronize(B.cap));
    }
    wait_for_jobs(B, B.st);
    GM_CUDA(cudaGraphLaunch(B.exec, B.st));
    add_launches(B.graph_kernels);  // the engine and the collection kernel
    jobs_wait_for(B, B.st);
  });
}

map_status map_batch_results(map_batch* b, int64_t* J, int64_t* max_block_weight, int32_t* iters) {
  return batch_guard(b, [&](map_batch& B) {
    if (!B.tuned) throw ApiError(MAP_E_STATE, "map_batch_launch has not run");
    const size_t nj = B.jobs.size();
    GM_CUDA(cudaMemcpyAsync(B.h_res, B.d_res, sizeof(JobResult) * nj, cudaMemcpyDeviceToHost, B.st));
    GM_CUDA(cudaStreamSynchronize(B.st));
    bool capped = false;
    for (size_t i = 0; i < nj; i++) {
      if (J) J[i] = B.h_res[i].J;
      if (max_block_weight) max_block_weight[i] = B.h_res[i].maxw;
      if (iters) iters[i] = (int32_t)B.h_res[i].iters;
      B.jobs[i]->c.last_iters = (int32_t)B.h_res[i].iters;
      capped |= B.h_res[i].capped != 0;
    }
    if (capped) throw ApiError(MAP_E_TIMEOUT, "a job stopped at the iteration cap");
  });
}

map_status map_batch_schedule(const map_batch* b, int32_t* cluster, int32_t* tile_entries, int32_t* clusters,
                              double* tune_ms) {
  if (!b) return MAP_E_INVALID;
  if (!b->tuned) return MAP_E_STATE;
  if (cluster) *cluster = b->sched.C;
  if (tile_entries) *tile_entries = b->sched.te;
  if (clusters) *clusters = b->sched.ncl;
  if (tune_ms) *tune_ms = b->tune_ms;
  return MAP_OK;
}

const char* map_batch_last_error(const map_batch* b) {
  if (!b) return last_create_error().c_str();
  return b->err.c_str();
}

void map_batch_destroy(map_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->cap) cudaStreamSynchronize(b->cap);
  release(b);
  delete b;
}

}  // extern "C"
