/*
 * CPU oracle for the integrated multilevel process-mapping path
 * (GPU-IM, Section 4.2 of "GPU-Accelerated Algorithms for Process Mapping").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, serial, deliberately slow
 * restatement of what the mapping path computes, used to check the CUDA
 * library element by element.  Only the test-suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * All arithmetic is integer.  Graphs are CSR: xadj int64[n+1], adj int32[m],
 * adjw int32[m], vw int32[n]; both directions of every undirected edge are
 * stored with equal weight; rows are sorted ascending; no self-loops.
 * Mappings are PE ids in [0, k).
 *
 * Parity status: every function below is pinned by the tests (brute-force
 * enumeration, closed forms, invariants); the end-to-end solution quality of
 * the heuristic has no printed reference value in the paper ("parity
 * unpinned" as to quality; only its steps and invariants are pinned).
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

typedef struct {
  uint64_t seed;
  int32_t patience;          /* Alg. 6: 12 */
  int32_t weak_max;          /* Alg. 6: 2 weak rebalancing steps before a strong one */
  int32_t phi_num, phi_den;  /* Alg. 6: phi = 999/1000 */
  int32_t sigma_gap;         /* Section 4.2 rebalancing: sigma = L_max - 100 */
  int32_t coarsest_factor;   /* Section 4.2: coarsen until fewer than 8k vertices */
  int32_t cluster_iters;     /* label-propagation clustering iterations per level: 5 */
  int32_t cluster_cap_div;   /* cluster weight cap = L_max / 4 */
  int32_t max_levels;        /* 64 */
  int32_t stall_num, stall_den; /* stop coarsening if n_c > 9/10 n */
  int32_t coarsener;         /* 0: label-propagation clustering, 1: two-hop matching (Section 4.2) */
  int32_t match_rounds;      /* heavy-edge matching: at most this many rounds per level: 16 */
  int32_t initial;           /* mapping of the coarsest graph: 0: breadth-first chunks; 1: hierarchical
                                multisection (Section 4.2, initial partitioning) */
  int32_t lp_relax_num, lp_relax_den; /* Alg. 4 filter: 0 = non-negative gains only (the paper's);
                                          > 0: also -G < floor(num conn(v, P(v)) / den) (Jet's) */
  int32_t reb_objective;     /* rebalancing gain: 0 = edge cut (the paper's), 1 = Eq. 1's J gain */
} orc_params;

typedef struct {
  int32_t levels;            /* number of graphs in the hierarchy (>= 1) */
  int32_t n[65];
  int64_t m_dir[65];
  int64_t J[65];             /* J after refinement of each level */
  int32_t iters[65];         /* Alg. 6 iterations run on each level */
} orc_stats;

void orc_default_params(orc_params *p);

int64_t orc_dist(const int32_t *hier, const int32_t *dist, int32_t levels, int64_t p, int64_t q);
int64_t orc_num_pes(const int32_t *hier, int32_t levels);
int64_t orc_lmax(int64_t total_weight, int64_t k, double eps);

int64_t orc_objective(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                      const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                      const int32_t *pi, int64_t *block_weight /* k, may be NULL */,
                      int64_t *max_block_weight /* may be NULL */);

int64_t orc_gain(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                 const int32_t *hier, const int32_t *dist, int32_t levels, const int32_t *pi,
                 int32_t v, int32_t q);

int32_t orc_lp_step(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                    const int32_t *hier, const int32_t *dist, int32_t levels,
                    int32_t *pi, uint8_t *lock, int32_t *pi_prime, int64_t *gain,
                    uint8_t *in_x, uint8_t *moved);
int32_t orc_lp_step_relaxed(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                            const int32_t *hier, const int32_t *dist, int32_t levels,
                            int32_t *pi, uint8_t *lock, int32_t *pi_prime, int64_t *gain,
                            uint8_t *in_x, uint8_t *moved, int32_t relax_num, int32_t relax_den);

int32_t orc_rebalance(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                      const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                      int64_t lmax, int32_t strong, int32_t sigma_gap, uint64_t seed,
                      int32_t level, int32_t t, int32_t *pi, int32_t *dest, uint8_t *moved);
int32_t orc_rebalance_obj(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                          const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                          int64_t lmax, int32_t strong, int32_t sigma_gap, uint64_t seed,
                          int32_t level, int32_t t, int32_t *pi, int32_t *dest, uint8_t *moved,
                          int32_t objective);

int32_t orc_refine(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                   const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                   int64_t lmax, const orc_params *prm, int32_t level, int32_t rounds,
                   int32_t *pi, int64_t *out_J, int64_t *out_max_block_weight,
                   int32_t *trace_kind, int64_t *trace_J, int64_t *trace_maxw,
                   int32_t trace_cap);

int32_t orc_cluster(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                    const int32_t *vw, int64_t wcap, const orc_params *prm, int32_t level,
                    int32_t *M);

int32_t orc_match(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                  const int32_t *vw, int64_t lmax, const orc_params *prm, int32_t level, int32_t *mate,
                  int32_t *M, int32_t *stage_matched);

int64_t orc_contract(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                     const int32_t *vw, const int32_t *M, int32_t nc,
                     int64_t *xadj_c, int32_t *adj_c, int32_t *adjw_c, int32_t *vw_c);

void orc_initial(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                 int64_t k, int32_t *pi);

void orc_project(int32_t n, const int32_t *M, const int32_t *pi_coarse, int32_t *pi);

int64_t orc_map_run(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                    const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                    double eps, const orc_params *prm, int32_t *pi, orc_stats *stats);

uint64_t orc_hash(uint64_t seed, uint64_t x);

/* Hierarchical multisection (GPU-HM, Eq. 2, Alg. 2, Alg. 3). */
typedef struct {
  int64_t calls[16];     /* partitioner calls per hierarchy level (index i - 1) */
  double first_eps[16];  /* eps' of the first call at each level */
} orc_hm_stats;

double orc_adaptive_eps(double eps, int64_t cV, int64_t cVp, int64_t k, int64_t kp, int32_t d);

int32_t orc_build_subgraph(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                           const int32_t *vw, const int32_t *part, int32_t b, int64_t *xadj_s,
                           int32_t *adj_s, int32_t *adjw_s, int32_t *vw_s, int32_t *M, int64_t *out_m,
                           int64_t *out_w);

int64_t orc_hm_run(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                   const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                   double eps, const orc_params *prm, int32_t *pi, orc_hm_stats *stats);

#endif
