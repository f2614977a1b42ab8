// Host-side engine state of one mapping context (one task graph, one machine
// hierarchy) and the entry points of the refinement and coarsening engines.
#pragma once

#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/gpumap.h"
#include "common.cuh"
#include "prim.cuh"
#include "mid.cuh"

namespace gm {

struct CudaError : std::runtime_error {
  cudaError_t code;
  CudaError(cudaError_t c, const char* what, const char* file, int line)
      : std::runtime_error(std::string(cudaGetErrorString(c)) + " at " + file + ":" + std::to_string(line) +
                           " (" + what + ")"),
        code(c) {}
};
struct ApiError : std::runtime_error {
  map_status status;
  ApiError(map_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

constexpr int32_t kMaxRefineIters = (1 << 20) - 1;

// Step kinds of the Alg. 6 state machine.
enum : int32_t { KIND_LP = 0, KIND_WEAK = 1, KIND_STRONG = 2, KIND_NONE = 3 };

// Device-resident state of one Alg. 6 run.
struct RefineState {
  int64_t J;           // objective of the current mapping P'
  int64_t maxw;        // max block weight of P'
  int64_t best_J;      // objective of the best mapping P
  int64_t best_maxw;
  int32_t i;           // patience counter
  int32_t iw;          // consecutive weak rebalancing steps
  int32_t t;           // iterations started
  int32_t kind;        // step of the current iteration
  int32_t done;
  int32_t copy_best;   // the iteration just finished produced a new best
  int32_t rounds;      // >= 0: fixed number of iterations
  int32_t level;
  int32_t moved;       // vertices moved by the last step
  int32_t last_kind;   // kind of the iteration k_control just closed
  int32_t capped;      // the iteration cap ended the run
  int32_t pad2;
  unsigned long long kernels;  // kernels run by conditional graph bodies
};

// Device-resident state of the clustering loop of one level.
struct ClusterState {
  int32_t it;          // current iteration
  int32_t done;
  int64_t moved;       // vertices moved in the current iteration
  unsigned long long kernels;  // kernels run by conditional graph bodies
  int64_t ncont;       // contested requests of the current sub-round (appended)
};

// Kernel classes timed by the optional CUDA-event profiler.
enum : int32_t { PK_LP_GAIN = 0, PK_LP_AFTER = 1, PK_EVAL = 2, PK_CLUSTER = 3, PK_SORT = 4, PK_EVAL_CTL = 5,
                 PK_MATCH = 6, PK_CLUSTER_MID = 7, PK_CLUSTER_HIGH = 8, PK_EVAL_MID = 9, PK_EVAL_HIGH = 10,
                 PK_LP_GAIN_MID = 11, PK_LP_GAIN_HIGH = 12, PK_COUNT = 13 };

struct ProfRec {
  cudaEvent_t a, b;
  int32_t kind;
  int32_t level;
  int64_t bytes;
};

struct Level {
  int32_t n = 0;
  int64_t m = 0;
  int64_t* xadj = nullptr;
  int32_t* adj = nullptr;
  int32_t* adjw = nullptr;
  int32_t* vw = nullptr;
  int32_t* M = nullptr;        // fine -> coarse map (to level + 1)
  int32_t* pi = nullptr;       // mapping as PE codes
  int32_t* hi = nullptr;       // vertices of degree > kLowDeg, ascending
  int32_t n_hi = 0;
  int64_t m_hi = 0;            // CSR entries of the high-degree vertices
  int64_t m_huge = 0;          // CSR entries of the vertices of degree > mid_deg
  int32_t mid_deg = kMidDeg;   // warp-per-vertex bound of this level (autotuned, <= kMidDeg)
  int64_t split_req = kSplitDeg;  // hub split bound asked for (hub_split_deg: the one in force)
  int32_t tuned = 0;           // 1: (mid_deg, split_req) chosen by timing, 0: defaults or the config's
  int64_t max_deg = 0;         // largest degree (0 when n_hi == 0, i.e. at most kLowDeg)
  int32_t* huge = nullptr;     // positions in hi of the vertices of degree > kMidDeg, ascending
  int32_t n_huge = 0;
  int64_t* hi_off = nullptr;   // hash-table offsets of the high-degree vertices (n_hi + 1)
  int64_t hi_slots = 0;
  // the CSR entries of the vertices of degree > kMidDeg, flattened in huge[]
  // order and cut into chunks of kHubChunk entries (clustering):
  int64_t* hub_pre = nullptr;    // exclusive prefix of their degrees (n_huge + 1)
  int32_t* hub_chunk = nullptr;  // per chunk: the huge[] index of the row holding its first entry
  // per chunk, two slots (the large row holding its first entry, the large
  // row starting inside it): a clustering slice result, 16 bytes each
  unsigned long long* hub_part = nullptr;
  // rows of degree > hub_split_deg whose connectivity tables are summed over
  // chunks (LP gains, rebalancing selection): per huge[] row its index among
  // them (-1: rated whole), their list, and n_split x kc partial tables (zero
  // between uses)
  int64_t* hub_acc = nullptr;    // per huge[] row: a sum over chunks (zero between uses)
  int32_t* hub_sidx = nullptr;
  int32_t* hub_split = nullptr;
  int32_t* hub_gtab = nullptr;
  int32_t n_split = 0;
  int64_t hub_gtab_cap = 0;
  int64_t hub_split_deg = 0;
  int64_t hub_chunk_cap = 0;
  int64_t n_hub_chunks = 0;
  int32_t max_vw = 0;
  // instantiated Alg. 6 graph of this level and what it was captured for
  cudaGraphExec_t gexec = nullptr;
  int32_t g_rounds = -2;
  int32_t g_nhi = -1;
  int32_t g_nhuge = -1;
  long long g_root = 0;  // kernel nodes outside the conditional bodies
  // instantiated clustering graph of this level and its key
  cudaGraphExec_t cgexec = nullptr;
  int64_t cg_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long cg_root = 0;
};

// Device view of the flattened entries of the rows of degree > kMidDeg.
struct HubRows {
  const int32_t* __restrict__ hi;
  const int32_t* __restrict__ huge;
  int32_t n_huge;
  const int64_t* __restrict__ pre;    // n_huge + 1
  const int32_t* __restrict__ chunk;  // first row of each chunk
  int64_t nchunks;
};
inline HubRows hub_rows(const Level& L) {
  return HubRows{L.hi, L.huge, L.n_huge, L.hub_pre, L.hub_chunk, L.n_hub_chunks};
}

struct DevMem {
  map_alloc_fn afn = nullptr;
  map_free_fn ffn = nullptr;
  void* user = nullptr;
  cudaStream_t st = nullptr;
  struct Block {
    void* p;
    size_t bytes;
  };
  std::vector<Block> blocks;
  size_t total = 0;
  size_t peak = 0;  // largest `total` so far
  void* get(size_t bytes);
  void put(void* p);
  void release_all();
  template <class T>
  T* make(size_t count) {
    return static_cast<T*>(get(count * sizeof(T)));
  }
};

// statistics of the last hierarchical multisection run (hm.cu)
struct HmStats {
  int32_t levels = 0;
  int64_t calls[16] = {};
  double first_eps[16] = {};
  double ms_partition = 0, ms_build = 0, ms_total = 0;
  double ms_level[16] = {};                     // wall time of each level's partitioning
  double ms_create = 0, ms_run = 0, ms_destroy = 0;  // summed over the partitioner calls
  int32_t workers = 0;
};

struct Ctx;
// Takes the fused-engine refinements of contexts that run beside each other
// (a server's jobs) and runs them in shared launches of the engine, one
// thread-block cluster per job.  refine() returns once the level has been
// refined, with the job's final Alg. 6 state; the context's earlier work on
// its own stream is ordered before the launch and its later work after it.
struct EngineSink {
  virtual ~EngineSink() = default;
  virtual void refine(Ctx& c, int lvl, int32_t rounds, int C, RefineState* out) = 0;
};

struct Ctx {
  cudaStream_t st = nullptr;
  map_config cfg{};
  Topo topo{};
  int32_t k = 0;
  int64_t cV = 0;
  int64_t lmax = 0;
  double eps = 0;
  std::vector<int32_t> code_of_pe, pe_of_code;
  std::vector<int32_t> hier, dist;  // a_1..a_l, d_1..d_l as given
  HmStats hm;       // the last map_run_hm
  HmStats hm_init;  // the last initial mapping by hierarchical multisection
  int32_t* d_code_of_pe = nullptr;
  int32_t* d_pe_of_code = nullptr;
  std::vector<Level> lv;       // lv[0] = input graph
  int32_t n0 = 0;
  int64_t m0 = 0;
  DevMem mem;
  Capture cap;
  bool use_graphs = true;
  std::string err;
  int dev = 0;
  int num_sms = 0;
  size_t max_smem = 0;

  // refinement scratch (sized for level 0)
  int32_t* pp = nullptr;        // P'
  int64_t* gain = nullptr;
  uint8_t* inx = nullptr;
  uint8_t* lock = nullptr;      // moved by the last label-propagation step
  int32_t* pi_best = nullptr;
  int32_t* dest = nullptr;
  uint8_t* elig = nullptr;
  uint8_t* sel = nullptr;
  uint8_t* acc = nullptr;
  int64_t* sarr = nullptr;      // per-vertex prefix weights
  int64_t* W = nullptr;         // block weights [kc]
  int64_t* accepted = nullptr;  // [kc]
  int64_t* headP = nullptr;     // [kc]
  int64_t* Rb = nullptr;        // [kc + 1]
  int32_t* U = nullptr;         // [kc]
  int64_t* tab = nullptr;       // [kc * kBuckets] eligible weight per (block, bucket), zero between steps
  int32_t* bcut = nullptr;      // [kc] cut bucket per overloaded block
  int64_t* rem = nullptr;       // [kc] weight still to move inside the cut bucket
  int64_t* counters = nullptr;  // small device counters
  int64_t* Jacc = nullptr;
  unsigned int* evctr = nullptr;  // blocks finished in a fused J evaluation
  RefineState* state = nullptr;
  RefineState* h_state = nullptr;  // pinned mirror
  int64_t* h_small = nullptr;      // pinned, a few values read back together
  void* h_tables = nullptr;        // pinned staging of small PE code tables
  int64_t* d_stats = nullptr;      // device, per-level statistics
  int32_t* trace_kind = nullptr;
  int64_t* trace_J = nullptr;
  int64_t* trace_maxw = nullptr;
  int32_t trace_cap = 4096;
  int32_t last_iters = 0;
  // bumped by every coarsening (coarse level buffers may be freed and
  // reallocated): a batch built on this context refuses to launch after it
  uint64_t level_gen = 0;

  // sort / scan scratch
  SortBufs sort;
  ScanTmp scan;
  int64_t* P64 = nullptr;       // per-element prefix (max(m0, n0) + 1)
  int64_t* P64b = nullptr;

  // coarsening scratch
  int32_t* C = nullptr;         // cluster labels (int32, < 2 n0)
  int32_t* Wc = nullptr;        // cluster weights [n0]
  int32_t* ReqW = nullptr;      // requested weight per target [n0]
  int32_t* req = nullptr;       // requested target per vertex [n0]
  int32_t* rank = nullptr;      // label -> coarse id [2 n0 + 2]
  // chunk tickets of the hub clustering kernels: {next chunk, CTAs done},
  // zero between launches (the last CTA of a launch resets them)
  unsigned long long* hub_ctr = nullptr;
  // hash tables of the vertices of degree > kMidDeg during clustering: one
  // 64-bit word per slot, (label << 32) | summed weight, all slots empty
  // (~0) between sub-rounds
  unsigned long long* htab = nullptr;
  int64_t hcap = 0;
  bool htab_clean = false;
  uint32_t* errword = nullptr;
  ClusterState* cstate = nullptr;
  ClusterState* h_cstate = nullptr;  // pinned mirror
  void* mstate = nullptr;            // two-hop matching state (device)

  // fused small-level engine
  EngineSink* sink = nullptr;  // when set, runs the cluster-engine refinements (with other contexts')
  int eng_max_cluster = 0;
  void* eng_job = nullptr;    // device job descriptor
  void* gbar = nullptr;       // device barrier state of the grid-wide engine
  int eng_grid_blocks = 0;    // resident blocks of the grid-wide engine (0: not known yet)
  void* h_eng_job = nullptr;  // pinned staging

  // resident blocks per SM of a kernel (occupancy API, cached)
  std::unordered_map<const void*, int> occ;
  int resident_blocks(const void* fn, int threads, size_t smem) {
    auto it = occ.find(fn);
    if (it != occ.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) {
      cudaGetLastError();
      nb = 1;
    }
    occ[fn] = nb;
    return nb;
  }

  // profiler
  bool prof = false;
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  cudaEvent_t prof_begin();
  int32_t prof_level = 0;     // level of the launches being recorded
  void prof_end(cudaEvent_t a, int32_t kind, int64_t bytes);

  // stats
  double ms_coarsen = 0, ms_initial = 0, ms_refine = 0, ms_project = 0;
  double ms_tune = 0;             // host wall time the schedule autotuner spent
  RefineState* probe_state = nullptr;  // kind = LP, for the autotuner's timing probe
  int32_t iters[65] = {0};
  int32_t kinds[65][3] = {};  // map_run: LP, weak and strong iterations per level (from the trace)
  int64_t Jlev[65] = {0};
  double ms_level[65] = {0};
};

// api.cu: error text of the last failed context-free call on this thread
std::string& last_create_error();

// refine.cu
void refine_alloc(Ctx& c);
void compute_block_weights(Ctx& c, int lvl);
void objective(Ctx& c, int lvl, int64_t* J, int64_t* maxw);
int32_t lp_step(Ctx& c, int lvl);
int32_t rebalance_step(Ctx& c, int lvl, bool strong, int32_t t);
void refine(Ctx& c, int lvl, int32_t rounds, int64_t* J, int64_t* maxw, int32_t* iters);
void classify_degrees(Ctx& c, int lvl);

// Fused refinement engine (one cluster of CTAs per job), shared with the
// batch entry points.
int engine_max_clusters(int C, int te);  // resident clusters of C CTAs (0: not launchable)
size_t engine_job_bytes();
bool engine_job_write(Ctx& c, int lvl, int32_t rounds, void* dst);  // false: level unsuited to the engine
// whether a configuration uses the refinement variants (relaxed filter, J gains in rebalancing)
inline bool uses_variants(const map_config& cfg) { return cfg.lp_relax_num > 0 || cfg.reb_objective != 0; }
// var: some job uses the refinement variants (needs te = 512)
void engine_launch(cudaStream_t st, const void* d_jobs, int njobs, unsigned int* queue, int C, int te, int nclusters,
                   bool var);
bool barrier_selftest(cudaStream_t st);  // the bounded grid-barrier wait gives up and reports it
void drop_graph(Level& L);

// coarsen.cu
void coarsen_alloc(Ctx& c);
int32_t coarsen(Ctx& c);
void initial_map(Ctx& c);
void project(Ctx& c, int lvl);
void validate_graph(Ctx& c);

// the context's capture streams, created on first use
inline void cap_streams(Ctx& c) {
  for (auto& cs : c.cap.s)
    if (!cs) GM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
}

// initial.cu: breadth-first initial mapping of a large coarsest graph over the whole GPU; false when
// its component labelling did not settle within its round limit (the caller then runs the one-CTA kernel)
bool initial_map_large(Ctx& c);

// match.cu
int32_t match_level(Ctx& c, int lvl);  // two-hop matching of level lvl into its M; returns n_c

// hm.cu: hierarchical multisection of level lvl's graph into its pi (codes)
void hm_run(Ctx& c, int lvl, int32_t workers, HmStats* st);

}  // namespace gm

// The opaque handle of the C ABI.
struct map_ctx {
  gm::Ctx c;
};
