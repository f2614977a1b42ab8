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
void run_pipeline(Job& j, cudaStream_t stream) {
  const map_job& d = j.desc;
  map_ctx* ctx = nullptr;
  map_status st = map_create(d.xadj, d.adjncy, d.adjwgt, d.vwgt, d.n, j.hier.data(), j.dist.data(),
                             (int32_t)j.hier.size(), d.eps, j.has_cfg ? &j.cfg : nullptr, (void*)stream, 0, &ctx);
  if (st != MAP_OK) {
    fill_error(j.res, st, map_last_error(nullptr));
    return;
  }
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
        run_pipeline(*j, stream);
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
  if (S->opts.slots < 1 || S->opts.slots > 256 || S->opts.lookahead < 1 || S->opts.mem_budget < 0) {
    last_create_error() = "slots must be in [1, 256], lookahead >= 1, mem_budget >= 0";
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
  delete S;
}

}  // extern "C"
