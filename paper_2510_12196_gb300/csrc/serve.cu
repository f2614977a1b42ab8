// Mapping server: a request loop that admits jobs by device memory and runs
// the admitted ones concurrently, each on its own CUDA stream.
//
// `slots` worker threads take jobs from one queue.  A job is admissible when
// the device bytes estimated for the jobs already on the GPU plus its own fit
// in the memory budget (a job that alone exceeds the budget starts only when
// nothing else runs).  Admission looks at the first `lookahead` queued jobs,
// oldest first, so a small request can overtake a large one that does not fit
// yet; once the oldest job has been overtaken 4 x lookahead times, admission
// falls back to strict arrival order until it starts.  Every finished job
// returns its slot and its bytes and wakes the workers, so requests that
// arrive while others run are admitted as soon as slots and memory free up,
// and their kernels overlap with the running jobs' on the device.  A job is
// the ordinary pipeline (map_create, map_run, download of the mapping,
// map_destroy) on the worker's stream; its result is the one it has alone.
//
// Batching across requests: the small levels of the running jobs (those the
// fused engine refines on one thread-block cluster) are not launched by each
// job but handed to the server's level batcher, whose `batch_lanes` threads
// each take every refinement that is waiting when they become free and run
// them in one persistent launch of the engine, one cluster per job, largest
// job first; jobs asking for the same cluster size share a launch, the
// launches of one batch run side by side on the lane's streams.  While a
// batch runs, newly arriving refinements wait for the next free lane, so the
// batches grow with the load.  A job's result does not depend on the batch
// it ran in (the engine keeps each job's buffers), and by default the jobs
// leave out the cooperative whole-GPU engine, whose launches hold every SM
// and would stop the other jobs' kernels for their whole duration.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace gm {
namespace {

struct Job {
  uint64_t ticket = 0;
  map_job desc{};
  map_config cfg{};
  bool has_cfg = false;
  std::vector<int32_t> hier, dist;
  int64_t est = 0;
  int32_t skipped = 0;  // later jobs admitted before this one
  map_job_result res{};
  bool done = false;
};

int64_t code_space(const int32_t* hier, int32_t levels) {
  int bits = 0;
  for (int i = 0; i < levels; i++) {
    int b = 0;
    while (b < 31 && (1 << b) < hier[i]) b++;
    bits += b;
  }
  return bits > 30 ? (int64_t)1 << 30 : (int64_t)1 << bits;
}

// The server's level batcher (see the file comment).
class LevelBatcher final : public EngineSink {
 public:
  static constexpr int kMaxBatch = 256;
  static constexpr int kSizes = 5;  // cluster sizes 1, 2, 4, 8, 16

  struct Stats {
    int64_t launches = 0, jobs = 0;
    int32_t peak_batch = 0;
  };

  LevelBatcher(int dev, int lanes) : dev_(dev) {
    try {
      for (int i = 0; i < lanes; i++) lanes_.emplace_back(&LevelBatcher::lane, this);
    } catch (...) {
      stop();
      throw;
    }
  }
  ~LevelBatcher() override { stop(); }

  void refine(Ctx& c, int lvl, int32_t rounds, int C, RefineState* out) override {
    Req r;
    r.c = &c;
    r.lvl = lvl;
    r.rounds = rounds;
    r.C = C;
    GM_CUDA(cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming));
    const cudaError_t e = cudaEventRecord(r.ready, c.st);
    if (e != cudaSuccess) {
      cudaEventDestroy(r.ready);
      GM_CUDA(e);
    }
    {
      std::lock_guard<std::mutex> lock(mu_);
      pending_.push_back(&r);
    }
    cv_req_.notify_one();
    {
      std::unique_lock<std::mutex> lock(mu_);
      cv_done_.wait(lock, [&] { return r.done; });
    }
    cudaEventDestroy(r.ready);
    if (r.status != MAP_OK) throw ApiError(r.status, r.err);
    *out = r.st;
  }

  Stats stats() {
    std::lock_guard<std::mutex> lock(mu_);
    return stats_;
  }

 private:
  struct Req {
    Ctx* c = nullptr;
    int lvl = 0;
    int32_t rounds = 0;
    int C = 1;
    cudaEvent_t ready = nullptr;
    bool done = false;
    map_status status = MAP_OK;
    std::string err;
    RefineState st{};
  };

  void stop() {
    {
      std::lock_guard<std::mutex> lock(mu_);
      stopping_ = true;
    }
    cv_req_.notify_all();
    for (auto& t : lanes_)
      if (t.joinable()) t.join();
    lanes_.clear();
  }

  // One batch: the waiting requests grouped by cluster size, each group one
  // persistent launch on its own stream, largest job first.
  void run_batch(std::vector<Req*>& batch, cudaStream_t* st, void* d_jobs, unsigned int* d_queue,
                 unsigned char* h_jobs, RefineState* h_states) {
    const size_t jb = engine_job_bytes();
    std::vector<Req*> group[kSizes];
    for (Req* r : batch) {
      int g = 0;
      while (g + 1 < kSizes && (1 << g) < r->C) g++;
      group[g].push_back(r);
    }
    size_t off = 0;
    for (int g = 0; g < kSizes; g++) {
      std::vector<Req*>& rs = group[g];
      if (rs.empty()) continue;
      std::stable_sort(rs.begin(), rs.end(), [](const Req* x, const Req* y) {
        const Level& a = x->c->lv[x->lvl];
        const Level& b = y->c->lv[y->lvl];
        return (int64_t)a.n + a.m > (int64_t)b.n + b.m;
      });
      bool var = false;
      for (size_t i = 0; i < rs.size(); i++) {
        GM_CUDA(cudaStreamWaitEvent(st[g], rs[i]->ready, 0));
        if (!engine_job_write(*rs[i]->c, rs[i]->lvl, rs[i]->rounds, h_jobs + jb * (off + i)))
          throw ApiError(MAP_E_INTERNAL, "a level handed to the batcher does not suit the engine");
        var = var || uses_variants(rs[i]->c->cfg);
      }
      const int C = 1 << g;
      const int ncl = std::min<int>(engine_max_clusters(C, 512), (int)rs.size());
      if (ncl < 1) throw ApiError(MAP_E_CUDA, "the refinement engine cannot be launched on this device");
      unsigned char* dj = static_cast<unsigned char*>(d_jobs) + jb * off;
      GM_CUDA(cudaMemcpyAsync(dj, h_jobs + jb * off, jb * rs.size(), cudaMemcpyHostToDevice, st[g]));
      GM_CUDA(cudaMemsetAsync(d_queue + g, 0, sizeof(unsigned int), st[g]));
      engine_launch(st[g], dj, (int)rs.size(), d_queue + g, C, 512, ncl, var);
      for (size_t i = 0; i < rs.size(); i++)
        GM_CUDA(cudaMemcpyAsync(&h_states[off + i], rs[i]->c->state, sizeof(RefineState), cudaMemcpyDeviceToHost,
                                st[g]));
      {
        std::lock_guard<std::mutex> lock(mu_);
        stats_.launches++;
      }
      off += rs.size();
    }
    for (int g = 0; g < kSizes; g++) GM_CUDA(cudaStreamSynchronize(st[g]));
    off = 0;
    for (int g = 0; g < kSizes; g++)
      for (Req* r : group[g]) r->st = h_states[off++];
  }

  void lane() {
    cudaStream_t st[kSizes] = {};
    void* d_jobs = nullptr;
    unsigned int* d_queue = nullptr;
    unsigned char* h_jobs = nullptr;
    RefineState* h_states = nullptr;
    std::string setup_err;
    if (cudaSetDevice(dev_) != cudaSuccess) setup_err = "cudaSetDevice failed";
    for (int g = 0; g < kSizes && setup_err.empty(); g++)
      if (cudaStreamCreateWithFlags(&st[g], cudaStreamNonBlocking) != cudaSuccess) setup_err = "stream creation failed";
    if (setup_err.empty() && (cudaMalloc(&d_jobs, engine_job_bytes() * kMaxBatch) != cudaSuccess ||
                              cudaMalloc(&d_queue, kSizes * sizeof(unsigned int)) != cudaSuccess ||
                              cudaMallocHost(&h_jobs, engine_job_bytes() * kMaxBatch) != cudaSuccess ||
                              cudaMallocHost(&h_states, sizeof(RefineState) * kMaxBatch) != cudaSuccess))
      setup_err = "the level batcher could not allocate its buffers";
    if (!setup_err.empty()) cudaGetLastError();
    while (true) {
      std::vector<Req*> batch;
      {
        std::unique_lock<std::mutex> lock(mu_);
        cv_req_.wait(lock, [&] { return stopping_ || !pending_.empty(); });
        if (pending_.empty()) break;  // stopping
        while (!pending_.empty() && (int)batch.size() < kMaxBatch) {
          batch.push_back(pending_.front());
          pending_.pop_front();
        }
      }
      map_status status = MAP_OK;
      std::string err;
      if (!setup_err.empty()) {
        status = MAP_E_OOM;
        err = setup_err;
      } else {
        try {
          run_batch(batch, st, d_jobs, d_queue, h_jobs, h_states);
        } catch (const ApiError& e) {
          status = e.status;
          err = e.what();
        } catch (const CudaError& e) {
          status = e.code == cudaErrorMemoryAllocation ? MAP_E_OOM : MAP_E_CUDA;
          err = e.what();
        } catch (const std::exception& e) {
          status = MAP_E_INTERNAL;
          err = e.what();
        }
        if (status != MAP_OK)
          for (int g = 0; g < kSizes; g++) cudaStreamSynchronize(st[g]);
      }
      {
        std::lock_guard<std::mutex> lock(mu_);
        for (Req* r : batch) {
          r->status = status;
          r->err = err;
          r->done = true;
        }
        stats_.jobs += (int64_t)batch.size();
        stats_.peak_batch = std::max(stats_.peak_batch, (int32_t)batch.size());
      }
      cv_done_.notify_all();
    }
    for (int g = 0; g < kSizes; g++)
      if (st[g]) cudaStreamDestroy(st[g]);
    if (d_jobs) cudaFree(d_jobs);
    if (d_queue) cudaFree(d_queue);
    if (h_jobs) cudaFreeHost(h_jobs);
    if (h_states) cudaFreeHost(h_states);
    cudaGetLastError();
  }

  int dev_;
  std::mutex mu_;
  std::condition_variable cv_req_, cv_done_;
  std::deque<Req*> pending_;
  bool stopping_ = false;
  Stats stats_;
  std::vector<std::thread> lanes_;
};

}  // namespace
}  // namespace gm

using namespace gm;

struct map_server {
  map_server_opts opts{};
  int dev = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_ticket = 1;
  int64_t bytes_in_flight = 0;
  int32_t running = 0;
  bool stopping = false;
  map_server_stats_t stats{};
  std::vector<std::thread> workers;
  std::unique_ptr<LevelBatcher> batcher;  // null: every job launches its own engine
  std::string err;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// The next admissible job (called with the lock held), removed from the queue.
Job* pick(map_server& S) {
  if (S.queue.empty() || S.running >= S.opts.slots) return nullptr;
  const int look = S.queue.front()->skipped >= 4 * S.opts.lookahead ? 1 : S.opts.lookahead;
  const int lim = std::min<int>(look, (int)S.queue.size());
  for (int i = 0; i < lim; i++) {
    Job* j = S.queue[i];
    if (S.running == 0 || S.bytes_in_flight + j->est <= S.opts.mem_budget) {
      for (int k = 0; k < i; k++) S.queue[k]->skipped++;
      S.queue.erase(S.queue.begin() + i);
      return j;
    }
  }
  return nullptr;
}

void fill_error(map_job_result& r, map_status st, const char* msg) {
  r.status = st;
  std::snprintf(r.error, sizeof(r.error), "%s", msg ? msg : "");
}

// The mapping pipeline of one job on `stream`.
void run_pipeline(map_server& S, Job& j, cudaStream_t stream) {
  const map_job& d = j.desc;
  map_config cfg;
  if (j.has_cfg) cfg = j.cfg;
  else map_config_default(&cfg);
  // the whole-GPU engine only where asked for explicitly (see the file comment)
  if (!S.opts.whole_gpu_levels && cfg.grid_engine_max_n == 0) cfg.grid_engine_max_n = -1;
  map_ctx* ctx = nullptr;
  map_status st = map_create(d.xadj, d.adjncy, d.adjwgt, d.vwgt, d.n, j.hier.data(), j.dist.data(),
                             (int32_t)j.hier.size(), d.eps, &cfg, (void*)stream, 0, &ctx);
  if (st != MAP_OK) {
    fill_error(j.res, st, map_last_error(nullptr));
    return;
  }
  ctx->c.sink = S.batcher.get();
  int64_t J = 0;
  st = map_run(ctx, d.out_pi, &J);
  if (st != MAP_OK) {
    fill_error(j.res, st, map_last_error(ctx));
  } else {
    map_stats_t s{};
    map_stats(ctx, &s);
    j.res.status = MAP_OK;
    j.res.J = J;
    j.res.levels = s.levels;
    j.res.device_bytes_peak = s.device_bytes_peak;
  }
  map_destroy(ctx);
}

void worker(map_server* S) {
  if (cudaSetDevice(S->dev) != cudaSuccess) cudaGetLastError();
  cudaStream_t stream = nullptr;
  if (!S->opts.runner) {
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      stream = nullptr;
    }
  }
  while (true) {
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait(lock, [&] { return S->stopping || (j = pick(*S)) != nullptr; });
      if (!j) break;  // stopping
      S->bytes_in_flight += j->est;
      S->running++;
      S->stats.running = S->running;
      S->stats.queued = (int64_t)S->queue.size();
      S->stats.bytes_in_flight = S->bytes_in_flight;
      S->stats.peak_bytes_in_flight = std::max(S->stats.peak_bytes_in_flight, S->bytes_in_flight);
      S->stats.peak_running = std::max(S->stats.peak_running, S->running);
      j->res.t_start_ms = S->now_ms();
    }
    if (S->opts.runner) {
      j->res.status = (map_status)S->opts.runner(&j->desc, (void*)stream, S->opts.runner_user, &j->res);
    } else {
      try {
        run_pipeline(*S, *j, stream);
      } catch (...) {
        fill_error(j->res, MAP_E_INTERNAL, "unexpected exception in the server worker");
      }
    }
    {
      std::lock_guard<std::mutex> lock(S->mu);
      j->res.t_done_ms = S->now_ms();
      j->done = true;
      S->bytes_in_flight -= j->est;
      S->running--;
      S->stats.running = S->running;
      S->stats.bytes_in_flight = S->bytes_in_flight;
      if (j->res.status == MAP_OK) S->stats.completed++;
      else S->stats.failed++;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

void map_server_opts_default(map_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->slots = 8;
  o->lookahead = 8;
  o->batch_lanes = 0;
  o->whole_gpu_levels = 0;
}

int64_t map_job_estimate_bytes(int32_t n, int64_t m_dir, const int32_t* hier, int32_t levels) {
  if (n < 0 || m_dir < 0 || !hier || levels < 1 || levels > 16) return -1;
  const int64_t cap = std::max<int64_t>({m_dir, (int64_t)n, 1});
  const int64_t kc = code_space(hier, levels);
  // sort buffers and prefix arrays (40 B per entry of the larger of n and
  // m_dir); the input graph and its coarser levels (up to twice the input's
  // entries, as on degree-skewed graphs that coarsen slowly), with the hash
  // tables of high-degree vertices (56 B per CSR entry together); per-vertex
  // clustering, refinement and level arrays (129 B per vertex); per-block
  // tables (560 B per PE code); traces and small buffers.
  return 40 * cap + 56 * m_dir + 129 * (int64_t)n + 560 * kc + (2 << 20);
}

map_status map_server_create(const map_server_opts* opts, map_server** out) {
  if (!out) return MAP_E_INVALID;
  *out = nullptr;
  std::unique_ptr<map_server> S(new (std::nothrow) map_server());
  if (!S) return MAP_E_OOM;
  if (opts) S->opts = *opts;
  else map_server_opts_default(&S->opts);
  if (S->opts.slots == 0) S->opts.slots = 8;
  if (S->opts.lookahead == 0) S->opts.lookahead = 8;
  if (S->opts.batch_lanes == 0) S->opts.batch_lanes = 2;
  if (S->opts.slots < 1 || S->opts.slots > 256 || S->opts.lookahead < 1 || S->opts.mem_budget < 0 ||
      S->opts.batch_lanes < -1 || S->opts.batch_lanes > 16 || S->opts.whole_gpu_levels < 0 ||
      S->opts.whole_gpu_levels > 1) {
    last_create_error() = "slots must be in [1, 256], lookahead >= 1, mem_budget >= 0, batch_lanes in -1..16, "
                          "whole_gpu_levels 0 or 1";
    return MAP_E_INVALID;
  }
  if (cudaGetDevice(&S->dev) != cudaSuccess) {
    cudaGetLastError();
    S->dev = 0;
  }
  if (S->opts.mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (!S->opts.runner && cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
      S->opts.mem_budget = (int64_t)(fr / 10 * 9);
    } else {
      cudaGetLastError();
      S->opts.mem_budget = (int64_t)1 << 40;
    }
  }
  S->t0 = std::chrono::steady_clock::now();
  if (!S->opts.runner && S->opts.batch_lanes > 0) {
    try {
      S->batcher.reset(new LevelBatcher(S->dev, S->opts.batch_lanes));
    } catch (...) {
      last_create_error() = "could not start the level batcher";
      return MAP_E_INTERNAL;
    }
  }
  try {
    for (int i = 0; i < S->opts.slots; i++) S->workers.emplace_back(worker, S.get());
  } catch (...) {
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    last_create_error() = "could not start the worker threads";
    return MAP_E_INTERNAL;
  }
  *out = S.release();
  return MAP_OK;
}

map_status map_server_submit(map_server* S, const map_job* job, uint64_t* ticket) {
  if (!S || !job || !ticket) return MAP_E_INVALID;
  if (job->n < 1 || !job->xadj || !job->hier || !job->dist || job->levels < 1 || job->levels > 16) {
    std::lock_guard<std::mutex> lock(S->mu);
    S->err = "job: n >= 1, xadj, hier and dist and 1..16 hierarchy levels are required";
    return MAP_E_INVALID;
  }
  std::unique_ptr<Job> j(new (std::nothrow) Job());
  if (!j) return MAP_E_OOM;
  j->desc = *job;
  j->hier.assign(job->hier, job->hier + job->levels);
  j->dist.assign(job->dist, job->dist + job->levels);
  if (job->cfg) {
    j->cfg = *job->cfg;
    j->has_cfg = true;
  }
  const int64_t m_dir = job->xadj[job->n];  // host CSR: the last offset is the entry count
  j->est = map_job_estimate_bytes(job->n, m_dir, job->hier, job->levels);
  j->res.device_bytes_est = j->est;
  j->res.user = job->user;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) {
      S->err = "the server is stopping";
      return MAP_E_STATE;
    }
    j->ticket = S->next_ticket++;
    j->res.ticket = j->ticket;
    j->res.t_submit_ms = S->now_ms();
    *ticket = j->ticket;
    S->queue.push_back(j.get());
    S->jobs.emplace(j->ticket, std::move(j));
    S->stats.submitted++;
    S->stats.queued = (int64_t)S->queue.size();
  }
  S->cv_work.notify_one();
  return MAP_OK;
}

map_status map_server_wait(map_server* S, uint64_t ticket, double timeout_ms, map_job_result* out) {
  if (!S) return MAP_E_INVALID;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) {
    S->err = "unknown or already collected ticket";
    return MAP_E_INVALID;
  }
  Job* j = it->second.get();
  auto ready = [&] { return j->done; };
  if (timeout_ms < 0) {
    S->cv_done.wait(lock, ready);
  } else if (!S->cv_done.wait_for(lock, std::chrono::duration<double, std::milli>(timeout_ms), ready)) {
    return MAP_E_TIMEOUT;
  }
  if (out) *out = j->res;
  S->jobs.erase(it);
  return MAP_OK;
}

map_status map_server_poll(map_server* S, uint64_t ticket, int32_t* done) {
  if (!S || !done) return MAP_E_INVALID;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) {
    S->err = "unknown or already collected ticket";
    return MAP_E_INVALID;
  }
  *done = it->second->done ? 1 : 0;
  return MAP_OK;
}

map_status map_server_stats(map_server* S, map_server_stats_t* out) {
  if (!S || !out) return MAP_E_INVALID;
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->stats;
  if (S->batcher) {
    const LevelBatcher::Stats b = S->batcher->stats();
    out->engine_launches = b.launches;
    out->engine_jobs = b.jobs;
    out->peak_batch = b.peak_batch;
  }
  out->queued = (int64_t)S->queue.size();
  out->mem_budget = S->opts.mem_budget;
  out->uptime_ms = S->now_ms();
  return MAP_OK;
}

const char* map_server_last_error(const map_server* S) {
  if (!S) return last_create_error().c_str();
  return S->err.c_str();
}

void map_server_destroy(map_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stopping = true;
    for (Job* j : S->queue) {  // queued jobs are cancelled
      fill_error(j->res, MAP_E_STATE, "cancelled: the server was destroyed");
      j->done = true;
    }
    S->queue.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& t : S->workers) t.join();
  S->batcher.reset();  // after the workers: their jobs may still hand it levels
  delete S;
}

}  // extern "C"
