/*
 * gpumap: GB300 (sm_103a) library for the integrated multilevel process
 * mapping method (GPU-IM, Section 4.2 of "GPU-Accelerated Algorithms for
 * Process Mapping", Samoldekin, Schulz & Woydt).
 *
 * The task graph G = (V, E) with vertex weights c and edge weights w is mapped
 * onto the k = a_1 * ... * a_l processing elements (PEs) of a hierarchical
 * machine H = a_1:...:a_l with distances D = d_1:...:d_l (Section 2).  The
 * library minimises the communication cost
 *     J(P) = sum over ordered pairs (u, v) in E of w(u, v) * D(P(u), P(v))
 * (Section 2; every undirected edge counts twice) under the balance bound
 *     c(V_b) <= L_max = ceil((1 + eps) c(V) / k)     for every PE b.
 * D(p, q) = 0 for p = q, else d_i for the smallest level i whose group holds
 * both; PE p lies in level-i group floor(p / (a_1 ... a_i)), so PEs p and p+1
 * share a processor when a_1 > 1.
 *
 * Conventions shared by every call:
 *  - Graphs are CSR: xadj int64[n+1], adjncy int32[m], adjwgt int32[m],
 *    vwgt int32[n].  Both directions of every edge are stored with equal
 *    weight, each row is strictly ascending (no duplicates), no self-loops,
 *    all weights >= 1, sum of vwgt < 2^31 and sum of adjwgt < 2^31.
 *  - Mappings are int32 PE ids in [0, k), one per vertex.
 *  - Host pointers unless stated otherwise.  The caller keeps ownership of
 *    every buffer it passes; map_create copies its inputs.  The library owns
 *    all device memory of a context and frees it in map_destroy.
 *  - Work is enqueued on the CUDA stream given to map_create.  Calls that
 *    return host data synchronise that stream before returning.
 *  - Every call returns a map_status; on error map_last_error gives a text.
 *    No C++ exception crosses this interface.
 *  - Results are deterministic: the same inputs and seed give bit-identical
 *    mappings and objectives on every run, whatever the launch schedule.
 */
#ifndef GPUMAP_H
#define GPUMAP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GPUMAP_API __attribute__((visibility("default")))
#else
#define GPUMAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct map_ctx map_ctx;

typedef enum {
  MAP_OK = 0,
  MAP_E_INVALID = 1,   /* malformed argument or graph (see map_last_error) */
  MAP_E_OOM = 2,       /* device allocation failed */
  MAP_E_CUDA = 3,      /* a CUDA call failed */
  MAP_E_OVERFLOW = 4,  /* weight sums exceed the int32 contract */
  MAP_E_TIMEOUT = 5,   /* a bounded device wait gave up */
  MAP_E_STATE = 6,     /* call made in the wrong state (e.g. level not built) */
  MAP_E_INTERNAL = 7   /* a device-side consistency check failed */
} map_status;

/* Optional device allocator: alloc returns device memory usable on `stream`
 * (NULL on failure); free releases it.  Used for every device buffer of a
 * context when both are set, else cudaMallocAsync / cudaFreeAsync are used;
 * then the device's default memory pool keeps up to 8 GiB of freed memory
 * for reuse (its release threshold, set once per process and device). */
typedef void* (*map_alloc_fn)(size_t bytes, void* user, void* stream);
typedef void (*map_free_fn)(void* ptr, size_t bytes, void* user, void* stream);

/* Tunable constants.  Defaults (map_config_default) are the paper's:
 * patience 12, weak_max 2, phi = 999/1000 (Alg. 6), sigma_gap 100 (Section
 * 4.2, rebalancing threshold sigma = L_max - 100), coarsest_factor 8
 * (coarsen until fewer than 8k vertices, Section 4.2, initial partitioning);
 * cluster_iters 5, cluster_cap_div 4, max_levels 64 and stall 9/10 belong to
 * the label-propagation clustering coarsener; match_rounds 16 to the two-hop
 * matching coarsener (Section 4.2, "Matching"). */
typedef struct {
  uint64_t seed;
  int32_t patience;
  int32_t weak_max;
  int32_t phi_num, phi_den;
  int32_t sigma_gap;
  int32_t coarsest_factor;
  int32_t cluster_iters;
  int32_t cluster_cap_div;
  int32_t max_levels;
  int32_t stall_num, stall_den;
  map_alloc_fn alloc;
  map_free_fn free;
  void* alloc_user;
  int32_t launch_mode;   /* 0: refinement and clustering loops as CUDA graphs (default); 1: stream launches */
  int32_t engine_max_n;  /* levels with at most this many vertices are refined by the fused one-launch
                            engine on one thread-block cluster (rows of degree > 128 by whole CTAs; a level
                            with such a row needs a PE code space whose connectivity table, conn per code
                            plus the level group sums, fits in 96 KiB); 0: library default (32768); -1: never */
  int32_t grid_engine_max_n; /* larger levels with at most this many vertices (same condition) run the same
                            engine over all SMs (cooperative launch); 0: library default (262144); -1: never */
  int32_t coarsener;     /* 0: label-propagation clustering (default); 1: two-hop matching (heavy-edge rounds
                            with the rating w^2 / (c(u) c(v)), then leaf, twin, relative and isolated pairing
                            while at most 75% of the vertices are matched) */
  int32_t match_rounds;  /* heavy-edge matching rounds at most (each matches mutual preferences; stops early
                            when a round matches nothing) */
  int32_t initial;       /* mapping of the coarsest graph: 0: breadth-first chunks (default); 1: hierarchical
                            multisection (as map_run_hm, on the coarsest graph, its partitioner starting
                            from breadth-first chunks; Section 4.2, initial partitioning) */
  int32_t lp_relax_num;  /* Alg. 4 filter.  0 (default): only moves of gain G >= 0 enter X, as in the paper;
                            > 0: also moves with -G < floor(lp_relax_num conn(v, P(v)) / lp_relax_den),
                            conn(v, P(v)) = weight of v's edges inside its PE (the filter Section 4.2
                            describes for Jet) */
  int32_t lp_relax_den;  /* >= 1 (default 1) */
  int32_t reb_objective; /* rebalancing gains: 0 (default): edge cut conn(v, q) - conn(v, P(v)), as the paper
                            settles on; 1: Eq. 1's J gain G_q(v) for the destination choice and the loss
                            buckets (the variant Section 4.2 reports trying) */
  int32_t mid_deg;       /* per-vertex split: vertices of degree 33..mid_deg get one warp each, larger ones the
                            hub kernels (chunks of their entries over the CTAs).  0 (default): chosen per
                            level by the autotuner (timing 255, 128 and 64 on levels whose rows of degree
                            > 32 hold at least 2^20 entries, else 255); 33..255: fixed */
  int32_t split_deg;     /* hub rows of more entries than this sum per-chunk connectivity tables over CTAs,
                            smaller ones are rated whole by one CTA.  0 (default): autotuned with mid_deg
                            (4096, 2048, 16384; else 4096); > 0: fixed */
} map_config;

typedef struct {
  int32_t levels;          /* graphs in the hierarchy (1 = not coarsened) */
  int32_t n[65];           /* vertices per level */
  int64_t m_dir[65];       /* CSR entries per level */
  int64_t J[65];           /* objective after refining each level (map_run) */
  int32_t iters[65];       /* Alg. 6 iterations per level (map_run) */
  double ms_coarsen, ms_initial, ms_refine, ms_project;  /* host wall time per phase */
  int64_t device_bytes;    /* device memory held by the context */
  int64_t device_bytes_peak; /* largest device memory the context has held */
  double ms_refine_level[65]; /* host wall time of Alg. 6 on each level (map_run; ends with a synchronisation) */
  int32_t mid_deg[65];     /* per-vertex split in force on each level (map_config.mid_deg) */
  int32_t split_deg[65];   /* hub split bound in force on each level (INT32_MAX: every hub row rated whole) */
  int32_t tuned[65];       /* 1: chosen by the autotuner; 0: defaults or the config's */
  double ms_tune;          /* host wall time the autotuner has spent on this context */
  int32_t lp_iters[65];    /* of iters[]: label-propagation, weak and strong rebalancing iterations per */
  int32_t weak_iters[65];  /* level (map_run; counted over the first 4096 iterations of a level) */
  int32_t strong_iters[65];
} map_stats_t;

/* Fills *cfg with the defaults listed above (seed 0x5EED0000, no allocator). */
GPUMAP_API void map_config_default(map_config* cfg);

/* Human-readable name of a status. */
GPUMAP_API const char* map_status_string(map_status s);

/* Creates a context for one graph and one hierarchy (Section 2).
 *  xadj, adjncy, adjwgt, vwgt: CSR as above; adjwgt / vwgt may be NULL
 *    (unit weights).  With inputs_on_device != 0 they are device pointers.
 *  n >= 1 vertices.
 *  hier[levels], dist[levels]: a_1..a_l (each >= 1) and d_1..d_l (each >= 0),
 *    1 <= levels <= 16; the PE code space prod 2^ceil(log2 a_i) must not
 *    exceed 16384 (k <= 16384 for power-of-two hierarchies).
 *  eps: imbalance, 0 <= eps < 1, quantised to parts per million.
 *  cfg: NULL for defaults.  stream: a cudaStream_t (NULL = legacy stream).
 * The graph is validated on the device (MAP_E_INVALID / MAP_E_OVERFLOW).
 * The initial mapping is all vertices on PE 0 until map_set_mapping or
 * map_initial / map_run set one.  *out receives the context. */
GPUMAP_API map_status map_create(const int64_t* xadj, const int32_t* adjncy, const int32_t* adjwgt,
                      const int32_t* vwgt, int32_t n, const int32_t* hier, const int32_t* dist,
                      int32_t levels, double eps, const map_config* cfg, void* stream,
                      int32_t inputs_on_device, map_ctx** out);

/* Frees all device memory of the context (after draining its stream). */
GPUMAP_API void map_destroy(map_ctx* ctx);

/* Text of the last error of this context (empty if none).  With ctx = NULL:
 * the error of the last failed map_create or map_objective_noalloc on the
 * calling thread. */
GPUMAP_API const char* map_last_error(const map_ctx* ctx);

/* Waits for all work of the context. */
GPUMAP_API map_status map_sync(map_ctx* ctx);

/* Number of PEs k and balance bound L_max of the context. */
GPUMAP_API map_status map_info(const map_ctx* ctx, int32_t* out_k, int64_t* out_lmax, int64_t* out_total_weight);

/* Sets / reads the mapping of hierarchy level `level` (0 = input graph):
 * pi is host int32[n_level] of PE ids in [0, k). */
GPUMAP_API map_status map_set_mapping(map_ctx* ctx, int32_t level, const int32_t* pi);
GPUMAP_API map_status map_get_mapping(map_ctx* ctx, int32_t level, int32_t* pi);

/* Objective J (Section 2, int64) and the maximum block weight (maxImb of
 * Alg. 6) of the current mapping of `level`.  Either output may be NULL. */
GPUMAP_API map_status map_objective(map_ctx* ctx, int32_t level, int64_t* out_J, int64_t* out_max_block_weight);

/* Block weights c(V_b), host int64[k], of the current mapping of `level`. */
GPUMAP_API map_status map_block_weights(map_ctx* ctx, int32_t level, int64_t* out_W);

/* One step of unconstrained label propagation (Alg. 4) on `level`:
 * gains by Eq. 1 over the neighbouring PEs, best target (lowest PE id on
 * ties), non-negative filter, recomputed gain under the ord approximation,
 * simultaneous move of the vertices that stay non-negative, and locking of
 * the moved vertices for the next label-propagation step (Section 4.2).
 * *out_moved (may be NULL) receives |M|. */
GPUMAP_API map_status map_lp_step(map_ctx* ctx, int32_t level, int32_t* out_moved);

/* The per-vertex results of the last map_lp_step on `level` (host arrays of
 * n_level entries, any may be NULL): target PE P'(v) (P(v) outside X),
 * gain g(v) (0 outside X), membership in X, and the lock (= moved) flags. */
GPUMAP_API map_status map_get_lp_state(map_ctx* ctx, int32_t level, int32_t* pi_prime, int64_t* gain,
                            uint8_t* in_x, uint8_t* moved);

/* Sets the lock flags (host uint8[n_level]) used by the next map_lp_step. */
GPUMAP_API map_status map_set_lock(map_ctx* ctx, int32_t level, const uint8_t* lock);

/* One weak (Alg. 5) or strong rebalancing step on `level` with edge-cut
 * loss (Section 4.2).  t is the iteration number that seeds the "random
 * block" fallback.  *out_moved (may be NULL) receives the moved count. */
GPUMAP_API map_status map_rebalance_step(map_ctx* ctx, int32_t level, int32_t strong, int32_t t, int32_t* out_moved);

/* Overall refinement (Alg. 6) of the current mapping of `level`.  rounds < 0
 * uses the patience rule (12 / 2 / phi); rounds >= 0 runs exactly that many
 * iterations.  The best mapping found is kept.  Outputs may be NULL. */
GPUMAP_API map_status map_refine(map_ctx* ctx, int32_t level, int32_t rounds, int64_t* out_J,
                      int64_t* out_max_block_weight, int32_t* out_iters);

/* Per-iteration record of the last map_refine (host arrays of `cap`
 * entries, any may be NULL): step kind (0 label propagation, 1 weak,
 * 2 strong), J and max block weight after the step. *out_count = iterations. */
GPUMAP_API map_status map_get_refine_trace(map_ctx* ctx, int32_t cap, int32_t* kind, int64_t* J,
                                int64_t* max_block_weight, int32_t* out_count);

/* Builds the coarse hierarchy (Section 4.2: coarsen until fewer than
 * coarsest_factor * k vertices) by label-propagation clustering and
 * contraction (summed vertex weights, fused parallel edges, dropped
 * self-loops; Section 2.1, Alg. 3).  Replaces any previous hierarchy. */
GPUMAP_API map_status map_coarsen(map_ctx* ctx, int32_t* out_levels);

/* Sizes of hierarchy level `level`. */
GPUMAP_API map_status map_level_info(map_ctx* ctx, int32_t level, int32_t* out_n, int64_t* out_m_dir);

/* Copies level `level` of the hierarchy to host arrays (any may be NULL):
 * CSR (xadj[n+1], adjncy[m], adjwgt[m], vwgt[n]) and the map M[n] of its
 * vertices to the next coarser level (undefined for the coarsest level). */
GPUMAP_API map_status map_get_level_graph(map_ctx* ctx, int32_t level, int64_t* xadj, int32_t* adjncy,
                               int32_t* adjwgt, int32_t* vwgt, int32_t* M);

/* Initial mapping of the coarsest level (breadth-first order cut into k
 * consecutive weight chunks; Section 4.2 leaves this partitioner open). */
GPUMAP_API map_status map_initial(map_ctx* ctx);

/* Uncontraction (Section 4.2): P_level(v) = P_{level+1}(M(v)). */
GPUMAP_API map_status map_project(map_ctx* ctx, int32_t level);

/* The whole GPU-IM pipeline: coarsen, initial mapping, Alg. 6 on the
 * coarsest level, then project and refine level by level.  out_pi (host
 * int32[n], may be NULL) receives the final mapping, *out_J its objective. */
GPUMAP_API map_status map_run(map_ctx* ctx, int32_t* out_pi, int64_t* out_J);

/* Statistics of the hierarchy and of the last map_run. */
/* Hierarchical multisection (GPU-HM; Section 4.1 "Hierarchical Multisection",
 * Eq. 2, Alg. 2, Alg. 3) of the context's input graph, instead of the
 * integrated pipeline of map_run.  From the top level a_l down, every
 * (sub)graph is partitioned into a_i blocks by the library's multilevel
 * pipeline on the one-level hierarchy a_i with distance 1 (its J is twice the
 * edge cut), under the adaptive imbalance of Eq. 2,
 *   eps' = ((1+eps) k' c(V) / (k c(V')))^(1/d) - 1,
 * k' = a_1...a_i, d = i, clamped to [0, 1 - 1e-6]; then the induced subgraph
 * of every block (Alg. 2, vertices renumbered in ascending id) is partitioned
 * one level down.  Block b at level i adds b * a_1...a_{i-1} to the PE id.
 * workers: host threads, each on its own stream, partitioning the subgraphs of
 * one level at the same time (0: 8); the result does not depend on it.
 * The mapping replaces the input level's (map_get_mapping, map_objective).
 * out_pi: host, n entries (may be NULL); out_J: J under the full hierarchy
 * (may be NULL).  Synchronises.  The partitioner contexts allocate with
 * cudaMallocAsync (a caller allocator in the config is not passed on).
 * Errors: MAP_E_INVALID (workers < 0, more than 16 levels), the partitioner's
 * status otherwise. */
GPUMAP_API map_status map_run_hm(map_ctx* ctx, int32_t workers, int32_t* out_pi, int64_t* out_J);

typedef struct {
  int32_t levels;          /* hierarchy levels */
  int32_t workers;         /* host threads used */
  int64_t calls[16];       /* partitioner calls at hierarchy level i (index i - 1), empty subgraphs skipped */
  double first_eps[16];    /* eps' of the first non-empty subgraph at each level */
  double ms_partition;     /* wall time in the partitioner calls */
  double ms_build;         /* wall time building the subgraphs (Alg. 2) */
  double ms_total;
  double ms_level[16];     /* wall time partitioning hierarchy level i (index i - 1) */
  double ms_create, ms_run, ms_destroy;  /* context setup, pipeline, teardown, summed over the calls */
} map_hm_stats_t;

/* Statistics of the last map_run_hm (which = 0) or of the last initial
 * mapping by hierarchical multisection inside map_run (which = 1,
 * map_config.initial = 1) on this context. */
GPUMAP_API map_status map_hm_stats(map_ctx* ctx, int32_t which, map_hm_stats_t* out);

GPUMAP_API map_status map_stats(map_ctx* ctx, map_stats_t* out);

/* Kernel classes of the optional profiler. */
enum {
  MAP_K_LP_GAIN = 0,   /* Alg. 4 step 1 (gains, low-degree path) */
  MAP_K_LP_AFTER = 1,  /* Alg. 4 step 2 (recomputed gains, low-degree path) */
  MAP_K_EVAL = 2,      /* objective J (low-degree path) */
  MAP_K_CLUSTER = 3,   /* clustering rating (low-degree path) */
  MAP_K_SORT = 4,      /* radix-sort scatter passes */
  MAP_K_EVAL_CTL = 5,  /* J evaluation launches that only close an LP or weak step (exact change of J
                          already accumulated): the controller, no CSR pass */
  MAP_K_MATCH = 6,     /* heavy-edge preference of the matching coarsener (one round) */
  MAP_K_CLUSTER_MID = 7,   /* clustering rating, one warp per vertex of degree 33..255 (bytes: the
                              active half of the rows, expected) */
  MAP_K_CLUSTER_HIGH = 8,  /* clustering rating, one CTA per vertex of degree > 255 (same model) */
  MAP_K_EVAL_MID = 9,      /* objective J, degree 33..255 */
  MAP_K_EVAL_HIGH = 10,    /* objective J, degree > 255 */
  MAP_K_LP_GAIN_MID = 11,  /* Alg. 4 step 1, degree 33..255 */
  MAP_K_LP_GAIN_HIGH = 12, /* Alg. 4 step 1, the vertices the per-warp tables do not take */
  MAP_K_COUNT = 13
};

/* Enables (1) or disables (0) CUDA-event timing of the kernel classes above
 * on the context's stream.  Timing adds two event records per timed launch
 * and no synchronisation. */
GPUMAP_API map_status map_profile_enable(map_ctx* ctx, int32_t enable);

/* Totals since the last read for kernel class `which` on hierarchy level
 * `level` (-1: all levels): timed launches, device time in ms (sum of event
 * intervals) and the algorithmic bytes those launches move by the library's
 * byte model (compulsory CSR and per-vertex streams; each neighbour gather
 * counted once as 4 bytes).  Synchronises the stream; the records read are
 * removed.  Outputs may be NULL. */
GPUMAP_API map_status map_profile_read(map_ctx* ctx, int32_t which, int32_t level, int64_t* launches,
                                       double* total_ms, int64_t* bytes);

/* Number of kernels this library has launched in this process so far. */
GPUMAP_API long long map_launch_count(void);

/* The paper has no counterpart to this call.  It returns what map_objective
 * returns (J and the maximum block weight) for callers that cannot or must
 * not allocate device memory: cudaMalloc / cudaFree may synchronise the whole
 * device and stall unrelated streams, and some callers run under a fixed
 * device-memory budget owned by their own pool, or just want the cost of a
 * mapping they already hold in device memory without creating a context.
 * It allocates nothing: no context, no cudaMalloc / cudaFree, no allocating
 * library routine.
 *  xadj, adjncy, adjwgt, vwgt, pi: DEVICE pointers (CSR as above, adjwgt may
 *    be NULL for unit weights; pi int32[n] PE ids in [0, k); entries out of
 *    range are skipped, not reported).  n >= 1.
 *  hier[levels], dist[levels]: HOST arrays as in map_create; the PE code
 *    space must not exceed 16384 (else MAP_E_INVALID, see map_last_error(NULL)).
 *  out: DEVICE int64[2], receives {J, maximum block weight}.
 *  stream: cudaStream_t; the work is enqueued on it and not waited for.
 * Scratch: one file-scope device array of about 192 KiB per device, held until
 * the process exits.  Every call shares it and it keeps the last call's
 * contents; each call clears what must start at zero.  Calls that overlap on
 * the GPU (several streams or host threads) race on it: serialise them.  The
 * first call on a device looks up the array's address with that device
 * current and keeps it for the process; make that first call before any
 * stream capture on the device.  A cudaDeviceReset invalidates the kept
 * address: do not call this entry point on a device after resetting it.
 * Rows are clamped to [0, xadj[n]): a malformed xadj cannot make it read
 * outside adjncy / adjwgt. */
GPUMAP_API map_status map_objective_noalloc(const int64_t* xadj, const int32_t* adjncy, const int32_t* adjwgt,
                                            const int32_t* vwgt, int32_t n, const int32_t* pi, const int32_t* hier,
                                            const int32_t* dist, int32_t levels, int64_t* out, void* stream);

/* Self-test of the engines' bounded waits (the paper has none: its
 * kernels do not wait on each other).  Launches, on `stream`, a cooperative
 * kernel whose grid barrier waits for one block more than the grid has, so
 * that every wait runs out after about a second; the blocks leave the kernel
 * and report it.  Returns MAP_E_TIMEOUT when the expiry was detected and
 * reported as designed (the device stays usable), MAP_E_INTERNAL if the
 * barrier was released or the expiry went unreported, MAP_E_CUDA on a CUDA
 * error.  The text is in map_last_error(NULL). */
GPUMAP_API map_status map_selftest_barrier_timeout(void* stream);

/* ------------------------------------------------------------------------
 * Batched refinement.  The paper refines one graph at a time; it has no
 * batched mode.  Here many contexts (graphs of uneven size, each with its own
 * hierarchy, distances and eps) are refined in ONE persistent kernel launch,
 * captured in a CUDA graph on the first map_batch_launch and replayed by
 * later ones: every job runs Alg. 6 on one level of its context (after
 * map_set_mapping, map_initial or map_project put a mapping there) from start
 * to end on one cluster of thread blocks, and the clusters take the jobs
 * largest first.  The result of each job is identical to map_refine(ctx,
 * level, rounds) on the same context, whatever the schedule.
 *
 * The schedule (CTAs per job and staged CSR entries per warp tile) is picked
 * by timing every candidate on the batch itself during the first launch (the
 * jobs' mappings are saved and restored around the trials) and cached per
 * batch shape for the rest of the process; autotune = 0 takes `cluster` and
 * `tile_entries` instead (0: a size-based default).
 *
 * Limits: all contexts on the current device, no context twice.  Rows of
 * degree > 128 are rated by whole CTAs from a connectivity table over the PE
 * codes in shared memory: a job whose refined level has such a row needs a
 * code space whose table (conn per code plus the level group sums, 4 bytes
 * each) fits in 96 KiB, e.g. every hierarchy of at most 8192 PEs
 * (MAP_E_INVALID otherwise: refine such a job with map_refine).  The batch keeps pointers into the contexts: destroy
 * it before them.  map_coarsen and map_run (which coarsens) may move a job's
 * level buffers: after either ran on a job, map_batch_launch returns
 * MAP_E_STATE; build a new batch.  The launch is asynchronous on the
 * stream given at creation; it waits for the jobs' pending work on their own
 * streams, and their later work waits for it.  map_batch_results
 * synchronises and returns the jobs' best J, maximum block weight and
 * iteration count in the order of `jobs`; afterwards map_get_mapping(job,
 * level) returns each job's refined mapping.  Errors of map_batch_create are
 * read with map_batch_last_error(NULL).
 * ------------------------------------------------------------------------ */
typedef struct map_batch map_batch;

typedef struct {
  int32_t level;         /* level refined in every job (0 = input graph) */
  int32_t rounds;        /* > 0: exactly that many Alg. 6 iterations; -1: Alg. 6 termination */
  int32_t autotune;      /* 1 (default): time the candidate schedules on the first launch */
  int32_t cluster;       /* autotune 0: CTAs per job, 1, 2, 4, 8 or 16; 0: size-based default */
  int32_t tile_entries;  /* autotune 0: staged CSR entries per warp tile, 256 or 512; 0: 512 */
} map_batch_opts;

/* level 0, rounds 10, autotune 1, the rest 0. */
GPUMAP_API void map_batch_opts_default(map_batch_opts* opts);
GPUMAP_API map_status map_batch_create(map_ctx* const* jobs, int32_t njobs, const map_batch_opts* opts,
                                       void* cuda_stream, map_batch** out);
GPUMAP_API map_status map_batch_launch(map_batch* batch);
/* Host arrays of njobs entries each (any may be NULL); MAP_E_TIMEOUT if a job
 * stopped at the iteration cap. */
GPUMAP_API map_status map_batch_results(map_batch* batch, int64_t* J, int64_t* max_block_weight, int32_t* iters);
/* The schedule in use (after the first launch): CTAs per job, staged entries
 * per warp tile, clusters in the persistent grid, and the wall time the
 * autotuner spent (0 when the schedule came from the cache or the options). */
GPUMAP_API map_status map_batch_schedule(const map_batch* batch, int32_t* cluster, int32_t* tile_entries,
                                         int32_t* clusters, double* tune_ms);
GPUMAP_API const char* map_batch_last_error(const map_batch* batch);
GPUMAP_API void map_batch_destroy(map_batch* batch);

/* ------------------------------------------------------------------------
 * Serving.  The paper maps one graph per program run; it has no serving
 * mode.  A server runs a request loop: submitted jobs wait in a queue and are
 * admitted by device memory; `slots` worker threads, each with its own CUDA
 * stream, run the admitted jobs concurrently, so a request that arrives while
 * others are on the GPU starts as soon as a slot and memory are free and its
 * kernels overlap with theirs (continuous batching).  The jobs' small levels
 * are batched across requests: each refinement that the fused engine would
 * run on one thread-block cluster waits for a free batcher lane, which runs
 * every waiting refinement in one persistent engine launch (one cluster per
 * job, largest first), so batches grow with the load.  A job is admissible
 * when the estimated device bytes of the running jobs plus its own
 * (map_job_estimate_bytes) fit in `mem_budget`; a job that alone exceeds the
 * budget starts only when nothing else runs.  Admission examines the oldest
 * `lookahead` queued jobs in arrival order, so a small job may overtake a
 * large one that does not fit yet; after the oldest job has been overtaken
 * 4 x lookahead times, admission is in strict arrival order until it starts.
 * A job is the whole pipeline: map_create from host buffers, map_run,
 * download of the mapping, map_destroy; its result equals the one it has
 * when run alone.  The job's host buffers are read while it runs: keep them
 * valid until map_server_wait returns it.  All calls are thread-safe; do not
 * call any of them on a server after map_server_destroy.
 * ------------------------------------------------------------------------ */
typedef struct map_server map_server;

typedef struct {
  const int64_t* xadj;        /* host CSR as for map_create (inputs_on_device = 0) */
  const int32_t* adjncy;
  const int32_t* adjwgt;      /* NULL: unit weights */
  const int32_t* vwgt;        /* NULL: unit weights */
  int32_t n;
  const int32_t* hier;        /* copied at submission */
  const int32_t* dist;        /* copied at submission */
  int32_t levels;
  double eps;
  const map_config* cfg;      /* copied at submission; NULL: map_config_default */
  int32_t* out_pi;            /* host, n entries (PE ids); NULL: not downloaded */
  void* user;                 /* returned in the result */
} map_job;

typedef struct {
  uint64_t ticket;
  map_status status;          /* of the job's pipeline */
  int32_t levels;
  int64_t J;
  int64_t device_bytes_est;   /* estimate used for admission */
  int64_t device_bytes_peak;  /* what the job's context held at most */
  double t_submit_ms, t_start_ms, t_done_ms;  /* milliseconds since map_server_create */
  void* user;
  char error[256];
} map_job_result;

/* Replaces the pipeline of every job (a dry run, or a test of the request
 * loop without a GPU): called on a worker thread with the worker's stream
 * (NULL when a runner is set); returns the job's status and may fill J and
 * levels of *out. */
typedef int32_t (*map_job_runner)(const map_job* job, void* stream, void* user, map_job_result* out);

typedef struct {
  int32_t slots;              /* jobs running at once (worker threads); 0: 8 */
  int32_t lookahead;          /* queued jobs examined for admission; 0: 8 (1: strict arrival order) */
  int64_t mem_budget;         /* device bytes for the running jobs; 0: 90% of the free memory at creation */
  map_job_runner runner;      /* NULL: the mapping pipeline */
  void* runner_user;
  int32_t batch_lanes;        /* small levels of the running jobs (those the fused engine refines on one
                                 cluster) are refined together, in shared engine launches by this many
                                 batcher threads; 0: 2; -1: each job launches its own engine */
  int32_t whole_gpu_levels;   /* 0 (default): jobs whose config leaves grid_engine_max_n at 0 do not use the
                                 cooperative whole-GPU engine, whose launches hold every SM; 1: as configured */
} map_server_opts;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t queued, running;
  int64_t bytes_in_flight, peak_bytes_in_flight, mem_budget;
  int32_t peak_running;
  double uptime_ms;
  int64_t engine_launches;    /* launches of the level batcher */
  int64_t engine_jobs;        /* level refinements they ran */
  int32_t peak_batch;         /* most level refinements one batch took */
} map_server_stats_t;

/* slots 8, lookahead 8, mem_budget 0 (automatic), no runner, batch_lanes 0 (2), whole_gpu_levels 0. */
GPUMAP_API void map_server_opts_default(map_server_opts* opts);
/* Device bytes a job's context may hold (an upper estimate for graphs whose
 * coarser levels together hold at most twice the input's CSR entries, which
 * covers grids, geometric and R-MAT graphs); -1 on bad arguments. */
GPUMAP_API int64_t map_job_estimate_bytes(int32_t n, int64_t m_dir, const int32_t* hier, int32_t levels);
GPUMAP_API map_status map_server_create(const map_server_opts* opts, map_server** out);
GPUMAP_API map_status map_server_submit(map_server* server, const map_job* job, uint64_t* ticket);
/* Waits for the job (timeout_ms < 0: without limit; MAP_E_TIMEOUT when the
 * limit passes first), copies its result to *out and retires the ticket. */
GPUMAP_API map_status map_server_wait(map_server* server, uint64_t ticket, double timeout_ms, map_job_result* out);
GPUMAP_API map_status map_server_poll(map_server* server, uint64_t ticket, int32_t* done);
GPUMAP_API map_status map_server_stats(map_server* server, map_server_stats_t* out);
GPUMAP_API const char* map_server_last_error(const map_server* server);
/* Lets running jobs finish, cancels queued ones (status MAP_E_STATE), joins
 * the workers and frees the server. */
GPUMAP_API void map_server_destroy(map_server* server);

#ifdef __cplusplus
}
#endif

#endif /* GPUMAP_H */
