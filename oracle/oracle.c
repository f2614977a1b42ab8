/*
 * CPU oracle for the integrated multilevel process-mapping path.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h): a plain serial restatement of
 * Section 4.2 of "GPU-Accelerated Algorithms for Process Mapping" (GPU-IM)
 * with the deterministic readings listed per function.  No blocking, fusion
 * or reordering beyond what the definitions and algorithms state; the only
 * library primitive used is qsort.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>


/* ------------------------------------------------------------------------- */
/* Counter-based hash: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) applied  */
/* to the state seed ^ x.                                                     */
/* ------------------------------------------------------------------------- */
uint64_t orc_hash(uint64_t seed, uint64_t x) {
  uint64_t z = (seed ^ x) + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Hash streams.  Salt in bits 60..63, level above bit 32 (bit 52 for the   */
/* rebalancing stream, whose iteration counter t sits in bits 32..51).       */
static uint64_t h_active(uint64_t seed, int32_t level, int32_t v) {
  return orc_hash(seed, (1ULL << 60) | ((uint64_t)level << 32) | (uint64_t)(uint32_t)v);
}
static uint64_t h_tie(uint64_t seed, int32_t level, int32_t t) {
  return orc_hash(seed, (2ULL << 60) | ((uint64_t)level << 32) | (uint64_t)(uint32_t)t);
}
static uint64_t h_rebalance(uint64_t seed, int32_t level, int32_t t, int32_t v) {
  return orc_hash(seed, (3ULL << 60) | ((uint64_t)level << 52) |
                            ((uint64_t)(t & 0xFFFFF) << 32) | (uint64_t)(uint32_t)v);
}
/* matching: noise of the edge {a, b} (a < b), and the hash of one neighbour */
/* (a neighbourhood hashes to the sum over its neighbours)                    */
static uint64_t h_edge(uint64_t seed, int32_t level, int32_t a, int32_t b) {
  return orc_hash(seed ^ ((4ULL << 60) | ((uint64_t)level << 48)), ((uint64_t)(uint32_t)a << 32) | (uint32_t)b);
}
static uint64_t h_nbr(uint64_t seed, int32_t u) {
  return orc_hash(seed, (5ULL << 60) | (uint64_t)(uint32_t)u);
}

void orc_default_params(orc_params *p) {
  p->seed = 0x5EED0000ULL;
  p->patience = 12;
  p->weak_max = 2;
  p->phi_num = 999;
  p->phi_den = 1000;
  p->sigma_gap = 100;
  p->coarsest_factor = 8;
  p->cluster_iters = 5;
  p->cluster_cap_div = 4;
  p->max_levels = 64;
  p->stall_num = 9;
  p->stall_den = 10;
  p->coarsener = 0;
  p->match_rounds = 16;
  p->initial = 0;
  p->lp_relax_num = 0;
  p->lp_relax_den = 1;
  p->reb_objective = 0;
}

/* ------------------------------------------------------------------------- */
/* Section 2: hierarchy H = a_1:...:a_l, k = prod a_i, distances d_1:...:d_l. */
/* PE p lies in level-i group floor(p / (a_1...a_i)); two different PEs have  */
/* cost d_i for the smallest level i whose group contains both (d_1: same     */
/* processor, d_2: same node, ...).  D(p, p) = 0.                             */
/* ------------------------------------------------------------------------- */
int64_t orc_num_pes(const int32_t *hier, int32_t levels) {
  int64_t k = 1;
  for (int i = 0; i < levels; i++) k *= hier[i];
  return k;
}

int64_t orc_dist(const int32_t *hier, const int32_t *dist, int32_t levels, int64_t p, int64_t q) {
  if (p == q) return 0;
  int64_t group_size = 1;
  for (int i = 0; i < levels; i++) {
    group_size *= hier[i];
    if (p / group_size == q / group_size) return dist[i];
  }
  return dist[levels - 1]; /* unreachable for p, q in [0, k) */
}

/* Section 2: L_max = ceil((1 + eps) c(V) / k), eps quantised to parts per   */
/* million so that the bound is an exact integer ceiling.                    */
int64_t orc_lmax(int64_t total_weight, int64_t k, double eps) {
  double scaled = eps * 1e6;
  int64_t e = (int64_t)(scaled < 0 ? scaled - 0.5 : scaled + 0.5);
  int64_t num = (1000000 + e) * total_weight;
  int64_t den = 1000000 * k;
  return (num + den - 1) / den;
}

/* ------------------------------------------------------------------------- */
/* Objective J (Section 2): sum over ordered pairs (i, j) of C_ij D_{P(i)P(j)}: */
/* every CSR entry contributes once, so each undirected edge counts twice.   */
/* Also the block weights c(V_b) and their maximum (maxImb of Alg. 6).       */
/* ------------------------------------------------------------------------- */
int64_t orc_objective(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                      const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                      const int32_t *pi, int64_t *block_weight, int64_t *max_block_weight) {
  int64_t J = 0;
  for (int32_t v = 0; v < n; v++)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
      J += (int64_t)adjw[e] * orc_dist(hier, dist, levels, pi[v], pi[adj[e]]);
  if (block_weight || max_block_weight) {
    int64_t k = orc_num_pes(hier, levels);
    int64_t *W = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    for (int32_t v = 0; v < n; v++) W[pi[v]] += vw[v];
    int64_t mx = 0;
    for (int64_t b = 0; b < k; b++) if (W[b] > mx) mx = W[b];
    if (block_weight) memcpy(block_weight, W, (size_t)k * sizeof(int64_t));
    if (max_block_weight) *max_block_weight = mx;
    free(W);
  }
  return J;
}

/* Eq. 1: G_q(v) = sum_{u in N(v)} w(v,u) (D(P(v), P(u)) - D(q, P(u))).      */
int64_t orc_gain(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                 const int32_t *hier, const int32_t *dist, int32_t levels, const int32_t *pi,
                 int32_t v, int32_t q) {
  (void)n;
  int64_t G = 0;
  for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
    int32_t b = pi[adj[e]];
    G += (int64_t)adjw[e] *
         (orc_dist(hier, dist, levels, pi[v], b) - orc_dist(hier, dist, levels, q, b));
  }
  return G;
}

/* Per-vertex connectivity (Section 4.2, last paragraph): conn(v, b) = sum of */
/* w(v,u) over neighbours u with P(u) = b.  Filled into a dense k-array; the  */
/* touched blocks are listed in first-seen order.                             */
typedef struct {
  int64_t *conn;   /* [k], all zero between uses */
  int32_t *list;   /* touched blocks */
  int32_t count;
} conn_table;

static void conn_fill(conn_table *t, const int64_t *xadj, const int32_t *adj,
                      const int32_t *adjw, const int32_t *pi, int32_t v) {
  t->count = 0;
  for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
    int32_t b = pi[adj[e]];
    if (t->conn[b] == 0) t->list[t->count++] = b;
    t->conn[b] += adjw[e];
  }
}
static void conn_clear(conn_table *t) {
  for (int32_t i = 0; i < t->count; i++) t->conn[t->list[i]] = 0;
  t->count = 0;
}

/* Eq. 1 regrouped by neighbouring block (identical sum in exact integers):  */
/* G_q(v) = sum_b conn(v,b) (D(P(v), b) - D(q, b)).                          */
static int64_t gain_from_conn(const conn_table *t, const int32_t *hier, const int32_t *dist,
                              int32_t levels, int32_t p, int32_t q) {
  int64_t G = 0;
  for (int32_t i = 0; i < t->count; i++) {
    int32_t b = t->list[i];
    G += t->conn[b] * (orc_dist(hier, dist, levels, p, b) - orc_dist(hier, dist, levels, q, b));
  }
  return G;
}

/* ------------------------------------------------------------------------- */
/* Alg. 4, unconstrained label propagation, one synchronous step over the    */
/* snapshot P (with move locking of Section 4.2: a vertex moved by the        */
/* previous label-propagation step is skipped).                               */
/*  1. every unlocked v: B = {P(u) : u in N(v)} without P(v); P'(v) = argmax */
/*     G_b(v) over B, ties to the lowest PE id; v in X iff G >= 0.            */
/*  2. every v in X: recompute the gain under the approximate future state   */
/*     given by ord: a neighbour u counts at P'(u) iff u in X and             */
/*     (g(u) > g(v) or (g(u) = g(v) and u < v)), else at P(u); v in M iff the */
/*     recomputed gain is >= 0.                                               */
/*  3. P(v) <- P'(v) for v in M, simultaneously; lock = indicator of M.       */
/* Vertices outside X report P'(v) = P(v), g(v) = 0.  Returns |M|.           */
/*                                                                           */
/* Relaxed filter (Section 4.2, the filter Jet uses; relax_num > 0): v also  */
/* enters X with a negative best gain G when -G < floor(c conn(v, P(v))),    */
/* c = relax_num / relax_den, conn(v, P(v)) the weight of v's edges into its */
/* own block.                                                                */
/* ------------------------------------------------------------------------- */
int32_t orc_lp_step(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                    const int32_t *hier, const int32_t *dist, int32_t levels,
                    int32_t *pi, uint8_t *lock, int32_t *pi_prime, int64_t *gain,
                    uint8_t *in_x, uint8_t *moved) {
  return orc_lp_step_relaxed(n, xadj, adj, adjw, hier, dist, levels, pi, lock, pi_prime, gain, in_x, moved, 0, 1);
}

int32_t orc_lp_step_relaxed(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                            const int32_t *hier, const int32_t *dist, int32_t levels,
                            int32_t *pi, uint8_t *lock, int32_t *pi_prime, int64_t *gain,
                            uint8_t *in_x, uint8_t *moved, int32_t relax_num, int32_t relax_den) {
  int64_t k = orc_num_pes(hier, levels);
  conn_table t;
  t.conn = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  t.list = (int32_t *)malloc((size_t)k * sizeof(int32_t));
  t.count = 0;

  /* step 1 */
  for (int32_t v = 0; v < n; v++) {
    pi_prime[v] = pi[v];
    gain[v] = 0;
    in_x[v] = 0;
    if (lock[v]) continue;
    conn_fill(&t, xadj, adj, adjw, pi, v);
    int32_t best_q = -1;
    int64_t best_g = 0;
    for (int32_t i = 0; i < t.count; i++) {
      int32_t b = t.list[i];
      if (b == pi[v]) continue;
      int64_t G = gain_from_conn(&t, hier, dist, levels, pi[v], b);
      if (best_q < 0 || G > best_g || (G == best_g && b < best_q)) {
        best_q = b;
        best_g = G;
      }
    }
    int64_t own = t.conn[pi[v]];
    conn_clear(&t);
    int admit = best_g >= 0;
    if (!admit && relax_num > 0) admit = -best_g < ((int64_t)relax_num * own) / relax_den;
    if (best_q >= 0 && admit) {
      in_x[v] = 1;
      pi_prime[v] = best_q;
      gain[v] = best_g;
    }
  }

  /* step 2 */
  for (int32_t v = 0; v < n; v++) {
    moved[v] = 0;
    if (!in_x[v]) continue;
    int64_t G = 0;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
      int32_t u = adj[e];
      int before = in_x[u] && (gain[u] > gain[v] || (gain[u] == gain[v] && u < v));
      int32_t beta = before ? pi_prime[u] : pi[u];
      G += (int64_t)adjw[e] * (orc_dist(hier, dist, levels, pi[v], beta) -
                               orc_dist(hier, dist, levels, pi_prime[v], beta));
    }
    if (G >= 0) moved[v] = 1;
  }

  /* step 3 */
  int32_t count = 0;
  for (int32_t v = 0; v < n; v++) {
    if (moved[v]) {
      pi[v] = pi_prime[v];
      count++;
    }
    lock[v] = moved[v];
  }
  free(t.conn);
  free(t.list);
  return count;
}

/* ------------------------------------------------------------------------- */
/* Alg. 5 (weak) and the strong variant, with the edge-cut loss that Section */
/* 4.2 settles on (its J-based variant is objective 1 below).                */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t a, b, c; int32_t v; } key4;

static int cmp_key4(const void *x, const void *y) {
  const key4 *p = (const key4 *)x, *q = (const key4 *)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  if (p->c != q->c) return p->c < q->c ? -1 : 1;
  if (p->v != q->v) return p->v < q->v ? -1 : 1;
  return 0;
}

/* log2-spaced loss buckets: "+" bucket for positive gain, "0" bucket for    */
/* zero gain, bucket 2 + floor(log2(-g)) for a negative gain g.              */
static int64_t loss_bucket(int64_t g) {
  if (g > 0) return 0;
  if (g == 0) return 1;
  int64_t x = -g, lg = 0;
  while (x > 1) { x >>= 1; lg++; }
  return 2 + lg;
}

int32_t orc_rebalance(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                      const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                      int64_t lmax, int32_t strong, int32_t sigma_gap, uint64_t seed,
                      int32_t level, int32_t t, int32_t *pi, int32_t *dest, uint8_t *moved) {
  return orc_rebalance_obj(n, xadj, adj, adjw, vw, hier, dist, levels, lmax, strong, sigma_gap, seed, level, t,
                           pi, dest, moved, 0);
}

/* objective 1 (Section 4.2 tried it: the rebalancing adapted to J): the     */
/* gain of moving v to b is Eq. 1's G_b(v) instead of the cut gain          */
/* conn(v, b) - conn(v, A); the destination is the neighbouring block below  */
/* sigma of largest G_b(v) (lowest id on ties), the random fallback's gain   */
/* is G_q(v) of the drawn block q, and buckets are taken of that gain.       */
int32_t orc_rebalance_obj(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                          const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                          int64_t lmax, int32_t strong, int32_t sigma_gap, uint64_t seed,
                          int32_t level, int32_t t, int32_t *pi, int32_t *dest, uint8_t *moved,
                          int32_t objective) {
  int64_t k = orc_num_pes(hier, levels);
  int64_t *W = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  int64_t cV = 0;
  for (int32_t v = 0; v < n; v++) { W[pi[v]] += vw[v]; cV += vw[v]; }

  /* destination threshold: sigma = L_max - gap (clamped below at the average */
  /* block weight) for weak rebalancing, L_max itself for the strong variant. */
  int64_t sigma;
  if (strong) {
    sigma = lmax;
  } else {
    int64_t avg = (cV + k - 1) / k;
    sigma = lmax - sigma_gap;
    if (sigma < avg) sigma = avg;
  }
  /* U: blocks that may receive a vertex, ascending (the "random block"     */
  /* fallback draws from it).                                                */
  int32_t *U = (int32_t *)malloc((size_t)k * sizeof(int32_t));
  int64_t nU = 0;
  for (int64_t b = 0; b < k; b++) if (W[b] <= sigma) U[nU++] = (int32_t)b;

  conn_table ct;
  ct.conn = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  ct.list = (int32_t *)malloc((size_t)k * sizeof(int32_t));
  ct.count = 0;

  int64_t *bucket = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  uint8_t *elig = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int32_t v = 0; v < n; v++) {
    dest[v] = pi[v];
    moved[v] = 0;
    int32_t A = pi[v];
    if (W[A] <= lmax) continue;                                  /* not overloaded */
    if (2 * k * (int64_t)vw[v] > 3 * (k * W[A] - cV)) continue;  /* heavy: > 1.5 (c(A) - c(V)/k) */
    conn_fill(&ct, xadj, adj, adjw, pi, v);
    int32_t best = -1;
    int64_t bestG = 0;
    for (int32_t i = 0; i < ct.count; i++) {
      int32_t b = ct.list[i];
      if (b == A || W[b] > sigma) continue;
      if (objective == 1) {
        int64_t G = gain_from_conn(&ct, hier, dist, levels, A, b);
        if (best < 0 || G > bestG || (G == bestG && b < best)) { best = b; bestG = G; }
      } else if (best < 0 || ct.conn[b] > ct.conn[best] || (ct.conn[b] == ct.conn[best] && b < best)) {
        best = b;
      }
    }
    int64_t g;
    if (best >= 0) {
      g = objective == 1 ? bestG : ct.conn[best] - ct.conn[A];
    } else {
      if (nU == 0) { conn_clear(&ct); continue; }
      best = U[h_rebalance(seed, level, t, v) % (uint64_t)nU];
      g = objective == 1 ? gain_from_conn(&ct, hier, dist, levels, A, best) : -ct.conn[A];
    }
    conn_clear(&ct);
    dest[v] = best;
    bucket[v] = loss_bucket(g);
    elig[v] = 1;
  }

  /* Per overloaded block A: eligible vertices in (bucket, id) order; v is    */
  /* selected iff the weight strictly before it is < c(A) - L_max.           */
  int32_t ne = 0;
  for (int32_t v = 0; v < n; v++) ne += elig[v];
  key4 *list = (key4 *)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(key4));
  ne = 0;
  for (int32_t v = 0; v < n; v++)
    if (elig[v]) { list[ne].a = pi[v]; list[ne].b = bucket[v]; list[ne].c = 0; list[ne].v = v; ne++; }
  qsort(list, (size_t)ne, sizeof(key4), cmp_key4);
  uint8_t *sel = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  {
    int64_t pre = 0;
    for (int32_t i = 0; i < ne; i++) {
      if (i == 0 || list[i].a != list[i - 1].a) pre = 0;
      int32_t v = list[i].v;
      if (pre < W[list[i].a] - lmax) sel[v] = 1;
      pre += vw[v];
    }
  }

  int32_t count = 0;
  if (!strong) {
    for (int32_t v = 0; v < n; v++)
      if (sel[v]) { pi[v] = dest[v]; moved[v] = 1; count++; }
  } else {
    /* Strong: movers grouped by destination in (bucket, id) order are        */
    /* accepted while the destination stays within L_max.                     */
    int32_t ns = 0;
    for (int32_t v = 0; v < n; v++)
      if (sel[v]) { list[ns].a = dest[v]; list[ns].b = bucket[v]; list[ns].c = 0; list[ns].v = v; ns++; }
    qsort(list, (size_t)ns, sizeof(key4), cmp_key4);
    int64_t *accepted = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    uint8_t *acc = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t inc = 0;
    for (int32_t i = 0; i < ns; i++) {
      if (i == 0 || list[i].a != list[i - 1].a) inc = 0;
      int32_t v = list[i].v;
      inc += vw[v];
      if (W[list[i].a] + inc <= lmax) { acc[v] = 1; accepted[list[i].a] += vw[v]; }
    }
    /* The rejected movers, in id order, are laid out on the residual room    */
    /* r(b) = L_max - c(b) - accepted(b) of the non-overloaded blocks in id   */
    /* order; a mover goes to the block whose room interval holds its whole   */
    /* weight interval [s, s + c(v)), otherwise it stays.                     */
    int64_t *room_start = (int64_t *)malloc((size_t)(k + 1) * sizeof(int64_t));
    int64_t *room = (int64_t *)malloc((size_t)k * sizeof(int64_t));
    room_start[0] = 0;
    for (int64_t b = 0; b < k; b++) {
      int64_t r = 0;
      if (W[b] <= lmax) { r = lmax - W[b] - accepted[b]; if (r < 0) r = 0; }
      room[b] = r;
      room_start[b + 1] = room_start[b] + r;
    }
    int64_t s = 0;
    for (int32_t v = 0; v < n; v++) {
      if (!sel[v]) continue;
      if (acc[v]) continue;
      for (int64_t b = 0; b < k; b++) {
        if (room[b] > 0 && room_start[b] <= s && s < room_start[b] + room[b]) {
          if (s + vw[v] <= room_start[b] + room[b]) { dest[v] = (int32_t)b; acc[v] = 1; }
          break;
        }
      }
      s += vw[v];
    }
    for (int32_t v = 0; v < n; v++) {
      if (sel[v] && acc[v]) { pi[v] = dest[v]; moved[v] = 1; count++; }
      else dest[v] = pi[v];
    }
    free(accepted); free(acc); free(room_start); free(room);
  }
  if (!strong)
    for (int32_t v = 0; v < n; v++) if (!sel[v]) dest[v] = pi[v];
  free(W); free(U); free(ct.conn); free(ct.list); free(bucket); free(elig); free(list); free(sel);
  return count;
}

/* ------------------------------------------------------------------------- */
/* Alg. 6, overall refinement: label propagation while balanced, else up to */
/* weak_max weak rebalancing steps followed by a strong one; the best        */
/* mapping is kept.  Readings: after a feasible move, the "better than the   */
/* best" test and the "better than phi times the best" test both compare     */
/* against the best J before the first of them replaces it; a feasible P'    */
/* always replaces an infeasible best (and resets the patience counter, as   */
/* a smaller maximum imbalance does).  rounds >= 0 runs exactly that many    */
/* iterations (no early exit); rounds < 0 uses the patience rule.            */
/* trace_kind records 0 = label                                              */
/* propagation, 1 = weak, 2 = strong per iteration; trace_J / trace_maxw the */
/* objective and maximum block weight after it.                              */
/* ------------------------------------------------------------------------- */
int32_t orc_refine(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                   const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                   int64_t lmax, const orc_params *prm, int32_t level, int32_t rounds,
                   int32_t *pi, int64_t *out_J, int64_t *out_max_block_weight,
                   int32_t *trace_kind, int64_t *trace_J, int64_t *trace_maxw,
                   int32_t trace_cap) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int32_t *cur = (int32_t *)malloc(nn * sizeof(int32_t));
  int32_t *pp = (int32_t *)malloc(nn * sizeof(int32_t));
  int32_t *dst = (int32_t *)malloc(nn * sizeof(int32_t));
  int64_t *gn = (int64_t *)malloc(nn * sizeof(int64_t));
  uint8_t *inx = (uint8_t *)malloc(nn);
  uint8_t *mv = (uint8_t *)malloc(nn);
  uint8_t *lock = (uint8_t *)calloc(nn, 1);
  memcpy(cur, pi, (size_t)n * sizeof(int32_t));

  int64_t best_maxw, best_J = orc_objective(n, xadj, adj, adjw, vw, hier, dist, levels, pi, NULL, &best_maxw);
  int32_t i = 0, iw = 0, t = 0;
  int64_t cur_maxw = best_maxw;
  while (1) {
    if (rounds >= 0) { if (t >= rounds) break; }
    else if (i >= prm->patience) break;
    i++;
    t++;
    int kind;
    if (cur_maxw <= lmax) {
      orc_lp_step_relaxed(n, xadj, adj, adjw, hier, dist, levels, cur, lock, pp, gn, inx, mv, prm->lp_relax_num,
                          prm->lp_relax_den);
      iw = 0;
      kind = 0;
    } else if (iw < prm->weak_max) {
      orc_rebalance_obj(n, xadj, adj, adjw, vw, hier, dist, levels, lmax, 0, prm->sigma_gap,
                    prm->seed, level, t, cur, dst, mv, prm->reb_objective);
      iw++;
      kind = 1;
    } else {
      orc_rebalance_obj(n, xadj, adj, adjw, vw, hier, dist, levels, lmax, 1, prm->sigma_gap,
                    prm->seed, level, t, cur, dst, mv, prm->reb_objective);
      iw = 0;
      kind = 2;
    }
    int64_t J = orc_objective(n, xadj, adj, adjw, vw, hier, dist, levels, cur, NULL, &cur_maxw);
    if (t - 1 < trace_cap) {
      if (trace_kind) trace_kind[t - 1] = kind;
      if (trace_J) trace_J[t - 1] = J;
      if (trace_maxw) trace_maxw[t - 1] = cur_maxw;
    }
    if (cur_maxw <= lmax) {
      if (best_maxw > lmax) {
        memcpy(pi, cur, (size_t)n * sizeof(int32_t));
        best_J = J; best_maxw = cur_maxw; i = 0;
      } else {
        int reset = (int64_t)prm->phi_den * J < (int64_t)prm->phi_num * best_J;
        if (J < best_J) {
          memcpy(pi, cur, (size_t)n * sizeof(int32_t));
          best_J = J; best_maxw = cur_maxw;
        }
        if (reset) i = 0;
      }
    } else if (cur_maxw < best_maxw) {
      memcpy(pi, cur, (size_t)n * sizeof(int32_t));
      best_J = J; best_maxw = cur_maxw; i = 0;
    }
  }
  if (out_J) *out_J = best_J;
  if (out_max_block_weight) *out_max_block_weight = best_maxw;
  free(cur); free(pp); free(dst); free(gn); free(inx); free(mv); free(lock);
  return t;
}

/* ------------------------------------------------------------------------- */
/* Coarsening by label-propagation clustering (the clustering alternative of */
/* Section 2.1 / Section 4.2).  Clusters start as singletons labelled by     */
/* vertex id.  Each iteration has two sub-rounds; v (with deg > 0) is active */
/* in sub-round bit(it) of its hash.  An active v rates every cluster of a   */
/* neighbour, and its own cluster, by the edge weight from v into it, picks  */
/* the best (ties: smaller tie-hash of the label, then smaller label) and    */
/* requests a move if that is another cluster with room under the cap.      */
/* Requests into one cluster are admitted in (hash, id) order while the      */
/* cluster stays within the cap (weights at the start of the sub-round).     */
/* Stop once fewer than 1% of the vertices moved in an iteration.  Then      */
/* isolated vertices are chunked in id order into clusters of weight <= cap */
/* (labelled n + chunk; a vertex straddling a chunk border stays alone).     */
/* M numbers the clusters by ascending label.  Returns n_c.                  */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t t; uint32_t h; int32_t v; } request;

static int cmp_request(const void *x, const void *y) {
  const request *p = (const request *)x, *q = (const request *)y;
  if (p->t != q->t) return p->t < q->t ? -1 : 1;
  if (p->h != q->h) return p->h < q->h ? -1 : 1;
  if (p->v != q->v) return p->v < q->v ? -1 : 1;
  return 0;
}

int32_t orc_cluster(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                    const int32_t *vw, int64_t wcap, const orc_params *prm, int32_t level,
                    int32_t *M) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t *C = (int64_t *)malloc(nn * sizeof(int64_t));      /* labels, may reach n + chunks */
  int64_t *Cs = (int64_t *)malloc(nn * sizeof(int64_t));
  int64_t *Wc = (int64_t *)malloc(nn * sizeof(int64_t));
  int64_t *Ws = (int64_t *)malloc(nn * sizeof(int64_t));
  int64_t *score = (int64_t *)calloc(nn, sizeof(int64_t));
  uint8_t *has = (uint8_t *)calloc(nn, 1);
  int32_t *touched = (int32_t *)malloc(nn * sizeof(int32_t));
  request *req = (request *)malloc(nn * sizeof(request));
  for (int32_t v = 0; v < n; v++) { C[v] = v; Wc[v] = vw[v]; }

  for (int32_t it = 0; it < prm->cluster_iters; it++) {
    int64_t moved = 0;
    for (int32_t r = 0; r < 2; r++) {
      memcpy(Cs, C, (size_t)n * sizeof(int64_t));
      memcpy(Ws, Wc, (size_t)n * sizeof(int64_t));
      int32_t nreq = 0;
      for (int32_t v = 0; v < n; v++) {
        if (xadj[v + 1] == xadj[v]) continue;
        if ((int32_t)((h_active(prm->seed, level, v) >> it) & 1ULL) != r) continue;
        int32_t nt = 0;
        int32_t own = (int32_t)Cs[v];
        has[own] = 1;
        touched[nt++] = own;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
          int32_t c = (int32_t)Cs[adj[e]];
          if (!has[c]) { has[c] = 1; touched[nt++] = c; }
          score[c] += adjw[e];
        }
        int32_t best = -1;
        for (int32_t i = 0; i < nt; i++) {
          int32_t c = touched[i];
          if (best < 0 || score[c] > score[best] ||
              (score[c] == score[best] &&
               (h_tie(prm->seed, level, c) < h_tie(prm->seed, level, best) ||
                (h_tie(prm->seed, level, c) == h_tie(prm->seed, level, best) && c < best))))
            best = c;
        }
        for (int32_t i = 0; i < nt; i++) { score[touched[i]] = 0; has[touched[i]] = 0; }
        if (best != own && Ws[best] + vw[v] <= wcap) {
          req[nreq].t = best;
          req[nreq].h = (uint32_t)(h_active(prm->seed, level, v) >> 32);
          req[nreq].v = v;
          nreq++;
        }
      }
      qsort(req, (size_t)nreq, sizeof(request), cmp_request);
      int64_t inc = 0;
      for (int32_t i = 0; i < nreq; i++) {
        if (i == 0 || req[i].t != req[i - 1].t) inc = 0;
        int32_t v = req[i].v;
        inc += vw[v];
        if (Ws[req[i].t] + inc <= wcap) {
          Wc[Cs[v]] -= vw[v];
          Wc[req[i].t] += vw[v];
          C[v] = req[i].t;
          moved++;
        }
      }
    }
    if (moved * 100 < (int64_t)n) break;
  }

  /* isolated vertices */
  int64_t s = 0;
  for (int32_t v = 0; v < n; v++) {
    if (xadj[v + 1] != xadj[v]) continue;
    int64_t first = s / wcap, last = (s + vw[v] - 1) / wcap;
    if (first == last) C[v] = (int64_t)n + first;
    s += vw[v];
  }

  /* number the clusters by ascending label */
  int64_t maxlabel = 2 * (int64_t)n + 1;
  int32_t *rank = (int32_t *)malloc((size_t)maxlabel * sizeof(int32_t));
  for (int64_t x = 0; x < maxlabel; x++) rank[x] = -1;
  for (int32_t v = 0; v < n; v++) rank[C[v]] = 0;
  int32_t nc = 0;
  for (int64_t x = 0; x < maxlabel; x++) if (rank[x] == 0) rank[x] = nc++;
  for (int32_t v = 0; v < n; v++) M[v] = rank[C[v]];
  free(C); free(Cs); free(Wc); free(Ws); free(score); free(has); free(touched); free(req); free(rank);
  return nc;
}

/* ------------------------------------------------------------------------- */
/* Coarsening by two-hop matching (Section 4.2, "Matching", after LaSalle et */
/* al. as used by Jet).                                                      */
/*                                                                           */
/* Heavy-edge rounds: every unmatched v with an unmatched neighbour u such   */
/* that c(v) + c(u) <= L_max prefers the u of largest rating                 */
/* exp*2 = w(v,u)^2 / (c(v) c(u)); ratings are compared exactly              */
/* (w1^2 c(u2) against w2^2 c(u1)), equal ratings by the smaller edge hash    */
/* (the deterministic noise), then the smaller u.  v and u are matched when  */
/* each prefers the other.  Rounds repeat until one matches nothing (at most */
/* match_rounds).                                                            */
/* While at most 75% of the vertices are matched, the two-hop stages follow, */
/* each on the still unmatched vertices, each pairing consecutive members of */
/* a group in (group, id) order (1st with 2nd, 3rd with 4th, ...; a pair     */
/* whose weight exceeds L_max stays unmatched), the 75% test repeated after  */
/* each: leaves (degree 1) grouped by their neighbour; twins (degree >= 2)   */
/* grouped by the top 31 bits of the hash of their neighbour set, paired     */
/* only if the sets are equal; relatives (degree >= 1) grouped by their      */
/* matchmaker, the neighbour                                                 */
/* of smallest (degree, id); isolated vertices (degree 0) in one group.      */
/* M numbers the pairs and single vertices by ascending smallest member.     */
/* mate[v] is v's partner or -1; stage_matched[0..5] (may be NULL) counts    */
/* the vertices matched by heavy edges, leaves, twins, relatives and        */
/* isolated pairing, and [5] the heavy-edge rounds run.  Returns n_c.        */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t g; int32_t v; } group_key;

static int cmp_group_key(const void *x, const void *y) {
  const group_key *p = (const group_key *)x, *q = (const group_key *)y;
  if (p->g != q->g) return p->g < q->g ? -1 : 1;
  if (p->v != q->v) return p->v < q->v ? -1 : 1;
  return 0;
}

static int same_neighbours(const int64_t *xadj, const int32_t *adj, int32_t a, int32_t b) {
  int64_t da = xadj[a + 1] - xadj[a], db = xadj[b + 1] - xadj[b];
  if (da != db) return 0;
  for (int64_t i = 0; i < da; i++)
    if (adj[xadj[a] + i] != adj[xadj[b] + i]) return 0;
  return 1;
}

/* pairs consecutive members of each group (keys sorted); returns matched */
static int64_t pair_groups(group_key *keys, int32_t cnt, const int32_t *vw, int64_t lmax, int twins,
                           const int64_t *xadj, const int32_t *adj, int32_t *mate) {
  int64_t matched = 0;
  qsort(keys, (size_t)cnt, sizeof(group_key), cmp_group_key);
  int32_t start = 0;
  for (int32_t i = 0; i < cnt; i++) {
    if (i > 0 && keys[i].g != keys[i - 1].g) start = i;
    if ((i - start) % 2 != 0) continue;               /* the first of a candidate pair */
    if (i + 1 >= cnt || keys[i + 1].g != keys[i].g) continue;
    int32_t a = keys[i].v, b = keys[i + 1].v;
    if ((int64_t)vw[a] + vw[b] > lmax) continue;
    if (twins && !same_neighbours(xadj, adj, a, b)) continue;
    mate[a] = b;
    mate[b] = a;
    matched += 2;
  }
  return matched;
}

int32_t orc_match(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                  const int32_t *vw, int64_t lmax, const orc_params *prm, int32_t level, int32_t *mate,
                  int32_t *M, int32_t *stage_matched) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int32_t *pref = (int32_t *)malloc(nn * sizeof(int32_t));
  group_key *keys = (group_key *)malloc(nn * sizeof(group_key));
  int64_t st[6] = {0, 0, 0, 0, 0, 0};
  for (int32_t v = 0; v < n; v++) mate[v] = -1;
  int64_t matched = 0;

  /* heavy-edge rounds */
  for (int32_t r = 0; r < prm->match_rounds; r++) {
    for (int32_t v = 0; v < n; v++) {
      pref[v] = -1;
      if (mate[v] >= 0) continue;
      int32_t best = -1;
      int64_t bw = 0;
      for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
        int32_t u = adj[e];
        if (mate[u] >= 0 || (int64_t)vw[v] + vw[u] > lmax) continue;
        int64_t w = adjw[e];
        int better;
        if (best < 0) {
          better = 1;
        } else {
          /* w^2 / c(u) against bw^2 / c(best) */
          unsigned __int128 lhs = (unsigned __int128)((uint64_t)(w * w)) * (uint64_t)vw[best];
          unsigned __int128 rhs = (unsigned __int128)((uint64_t)(bw * bw)) * (uint64_t)vw[u];
          if (lhs != rhs) {
            better = lhs > rhs;
          } else {
            uint64_t hu = h_edge(prm->seed, level, v < u ? v : u, v < u ? u : v);
            uint64_t hb = h_edge(prm->seed, level, v < best ? v : best, v < best ? best : v);
            better = hu < hb || (hu == hb && u < best);
          }
        }
        if (better) { best = u; bw = w; }
      }
      pref[v] = best;
    }
    int64_t now = 0;
    for (int32_t v = 0; v < n; v++) {
      int32_t u = pref[v];
      if (u >= 0 && pref[u] == v) { mate[v] = u; now++; }
    }
    matched += now;
    st[0] += now;
    st[5] = r + 1;
    if (now == 0) break;
  }

  /* two-hop stages while at most 75% are matched */
  for (int stage = 1; stage <= 4; stage++) {
    if (4 * matched > 3 * (int64_t)n) break;
    int32_t cnt = 0;
    for (int32_t v = 0; v < n; v++) {
      if (mate[v] >= 0) continue;
      int64_t d = xadj[v + 1] - xadj[v];
      uint64_t g;
      if (stage == 1) {          /* leaves */
        if (d != 1) continue;
        g = (uint64_t)(uint32_t)adj[xadj[v]];
      } else if (stage == 2) {   /* twins: the top 31 bits of the neighbour-set hash */
        if (d < 2) continue;
        g = 0;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) g += h_nbr(prm->seed, adj[e]);
        g >>= 33;
      } else if (stage == 3) {   /* relatives: the matchmaker */
        if (d < 1) continue;
        int32_t mm = -1;
        int64_t md = 0;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
          int32_t u = adj[e];
          int64_t du = xadj[u + 1] - xadj[u];
          if (mm < 0 || du < md || (du == md && u < mm)) { mm = u; md = du; }
        }
        g = (uint64_t)(uint32_t)mm;
      } else {                   /* isolated */
        if (d != 0) continue;
        g = 0;
      }
      keys[cnt].g = g;
      keys[cnt].v = v;
      cnt++;
    }
    int64_t got = pair_groups(keys, cnt, vw, lmax, stage == 2, xadj, adj, mate);
    matched += got;
    st[stage] = got;
  }

  /* number pairs and singles by their smallest member */
  int32_t nc = 0;
  for (int32_t v = 0; v < n; v++) {
    int32_t rep = (mate[v] >= 0 && mate[v] < v) ? mate[v] : v;
    if (rep == v) pref[v] = nc++;
  }
  for (int32_t v = 0; v < n; v++) {
    int32_t rep = (mate[v] >= 0 && mate[v] < v) ? mate[v] : v;
    M[v] = pref[rep];
  }
  if (stage_matched)
    for (int i = 0; i < 6; i++) stage_matched[i] = (int32_t)st[i];
  free(pref); free(keys);
  return nc;
}

/* ------------------------------------------------------------------------- */
/* Contraction (Section 2.1 and Alg. 3): every cluster becomes one coarse    */
/* vertex of summed weight; edges between different clusters are summed      */
/* into one coarse edge; edges inside a cluster (self-loops) are dropped.    */
/* Coarse rows ascending, adjacency ascending.  Returns the coarse m_dir.    */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t a, b, w; } triple;

static int cmp_triple(const void *x, const void *y) {
  const triple *p = (const triple *)x, *q = (const triple *)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return 0;
}

int64_t orc_contract(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                     const int32_t *vw, const int32_t *M, int32_t nc,
                     int64_t *xadj_c, int32_t *adj_c, int32_t *adjw_c, int32_t *vw_c) {
  for (int32_t x = 0; x < nc; x++) vw_c[x] = 0;
  for (int32_t v = 0; v < n; v++) vw_c[M[v]] += vw[v];
  int64_t m = xadj[n];
  triple *tr = (triple *)malloc((size_t)(m > 0 ? m : 1) * sizeof(triple));
  int64_t cnt = 0;
  for (int32_t v = 0; v < n; v++)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
      if (M[v] == M[adj[e]]) continue;
      tr[cnt].a = M[v]; tr[cnt].b = M[adj[e]]; tr[cnt].w = adjw[e]; cnt++;
    }
  qsort(tr, (size_t)cnt, sizeof(triple), cmp_triple);
  int64_t mc = 0;
  for (int32_t x = 0; x <= nc; x++) xadj_c[x] = 0;
  for (int64_t i = 0; i < cnt; i++) {
    if (mc > 0 && i > 0 && tr[i].a == tr[i - 1].a && tr[i].b == tr[i - 1].b) {
      adjw_c[mc - 1] += tr[i].w;
    } else {
      adj_c[mc] = tr[i].b;
      adjw_c[mc] = tr[i].w;
      xadj_c[tr[i].a + 1]++;
      mc++;
    }
  }
  for (int32_t x = 0; x < nc; x++) xadj_c[x + 1] += xadj_c[x];
  free(tr);
  return mc;
}

/* Uncontraction (Section 4.2): P(v) = P_coarse(M(v)).                       */
void orc_project(int32_t n, const int32_t *M, const int32_t *pi_coarse, int32_t *pi) {
  for (int32_t v = 0; v < n; v++) pi[v] = pi_coarse[M[v]];
}

/* ------------------------------------------------------------------------- */
/* Initial mapping of the coarsest graph (Section 4.2 leaves the partitioner */
/* open): breadth-first order from the lowest unvisited id (neighbours in    */
/* adjacency order), and a vertex whose preceding weight in that order is s  */
/* goes to PE floor(s k / c(V)), so consecutive PEs take consecutive chunks. */
/* ------------------------------------------------------------------------- */
void orc_initial(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                 int64_t k, int32_t *pi) {
  size_t nn = (size_t)(n > 0 ? n : 1);
  int32_t *queue = (int32_t *)malloc(nn * sizeof(int32_t));
  uint8_t *seen = (uint8_t *)calloc(nn, 1);
  int64_t cV = 0;
  for (int32_t v = 0; v < n; v++) cV += vw[v];
  int32_t tail = 0;
  for (int32_t s = 0; s < n; s++) {
    if (seen[s]) continue;
    int32_t head = tail;
    queue[tail++] = s;
    seen[s] = 1;
    while (head < tail) {
      int32_t v = queue[head++];
      for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
        int32_t u = adj[e];
        if (!seen[u]) { seen[u] = 1; queue[tail++] = u; }
      }
    }
  }
  int64_t pre = 0;
  for (int32_t i = 0; i < n; i++) {
    int32_t v = queue[i];
    pi[v] = (int32_t)(pre * k / cV);
    pre += vw[v];
  }
  free(queue); free(seen);
}

/* ------------------------------------------------------------------------- */
/* GPU-IM pipeline (Section 4.2): coarsen while n >= coarsest_factor * k     */
/* (stop on stall: n_c > 9/10 n, which is then discarded), map the coarsest */
/* graph, refine it with Alg. 6, then project and refine level by level.     */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  int64_t *xadj;
  int32_t *adj, *adjw, *vw, *M;
} level_graph;

int64_t orc_map_run(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                    const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                    double eps, const orc_params *prm, int32_t *pi, orc_stats *stats) {
  int64_t k = orc_num_pes(hier, levels);
  int64_t cV = 0;
  for (int32_t v = 0; v < n; v++) cV += vw[v];
  int64_t lmax = orc_lmax(cV, k, eps);
  level_graph *L = (level_graph *)calloc((size_t)prm->max_levels + 1, sizeof(level_graph));
  L[0].n = n;
  L[0].xadj = (int64_t *)xadj; L[0].adj = (int32_t *)adj; L[0].adjw = (int32_t *)adjw; L[0].vw = (int32_t *)vw;
  int32_t nl = 1;
  while (nl < prm->max_levels && (int64_t)L[nl - 1].n >= prm->coarsest_factor * k) {
    level_graph *f = &L[nl - 1];
    int64_t maxc = 0;
    for (int32_t v = 0; v < f->n; v++) if (f->vw[v] > maxc) maxc = f->vw[v];
    int64_t wcap = lmax / prm->cluster_cap_div;
    if (wcap < maxc) wcap = maxc;
    f->M = (int32_t *)malloc((size_t)(f->n > 0 ? f->n : 1) * sizeof(int32_t));
    int32_t nc;
    if (prm->coarsener == 1) {
      int32_t *mate = (int32_t *)malloc((size_t)(f->n > 0 ? f->n : 1) * sizeof(int32_t));
      nc = orc_match(f->n, f->xadj, f->adj, f->adjw, f->vw, lmax, prm, nl - 1, mate, f->M, NULL);
      free(mate);
    } else {
      nc = orc_cluster(f->n, f->xadj, f->adj, f->adjw, f->vw, wcap, prm, nl - 1, f->M);
    }
    if ((int64_t)nc * prm->stall_den > (int64_t)prm->stall_num * f->n) { free(f->M); f->M = NULL; break; }
    level_graph *c = &L[nl];
    c->n = nc;
    c->xadj = (int64_t *)malloc((size_t)(nc + 1) * sizeof(int64_t));
    int64_t mf = f->xadj[f->n];
    c->adj = (int32_t *)malloc((size_t)(mf > 0 ? mf : 1) * sizeof(int32_t));
    c->adjw = (int32_t *)malloc((size_t)(mf > 0 ? mf : 1) * sizeof(int32_t));
    c->vw = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    orc_contract(f->n, f->xadj, f->adj, f->adjw, f->vw, f->M, nc, c->xadj, c->adj, c->adjw, c->vw);
    nl++;
  }
  int32_t **P = (int32_t **)calloc((size_t)nl, sizeof(int32_t *));
  for (int32_t l = 0; l < nl; l++) P[l] = (int32_t *)malloc((size_t)(L[l].n > 0 ? L[l].n : 1) * sizeof(int32_t));
  int32_t top = nl - 1;
  if (prm->initial == 1) /* hierarchical multisection of the coarsest graph */
    orc_hm_run(L[top].n, L[top].xadj, L[top].adj, L[top].adjw, L[top].vw, hier, dist, levels, eps, prm,
               P[top], NULL);
  else
    orc_initial(L[top].n, L[top].xadj, L[top].adj, L[top].vw, k, P[top]);
  int64_t J = 0, maxw = 0;
  if (stats) { memset(stats, 0, sizeof(*stats)); stats->levels = nl; }
  for (int32_t l = top; l >= 0; l--) {
    if (l < top) orc_project(L[l].n, L[l].M, P[l + 1], P[l]);
    int32_t it = orc_refine(L[l].n, L[l].xadj, L[l].adj, L[l].adjw, L[l].vw, hier, dist, levels,
                            lmax, prm, l, -1, P[l], &J, &maxw, NULL, NULL, NULL, 0);
    if (stats && l <= 64) {
      stats->n[l] = L[l].n; stats->m_dir[l] = L[l].xadj[L[l].n]; stats->J[l] = J; stats->iters[l] = it;
    }
  }
  memcpy(pi, P[0], (size_t)n * sizeof(int32_t));
  for (int32_t l = 0; l < nl; l++) {
    free(P[l]);
    if (l > 0) { free(L[l].xadj); free(L[l].adj); free(L[l].adjw); free(L[l].vw); }
    free(L[l].M);
  }
  free(P); free(L);
  return J;
}

/* ------------------------------------------------------------------------- */
/* Hierarchical multisection (GPU-HM, Section 4.1 "Hierarchical             */
/* Multisection", Eq. 2, Alg. 2 and Alg. 3).                                 */
/*                                                                           */
/* Adaptive imbalance (Eq. 2): eps' = ((1+eps) k' c(V) / (k c(V')))^(1/d)-1, */
/* with k' the number of PEs the subgraph ends up on and d the number of     */
/* hierarchy levels still to partition, the current one included.           */
/* ------------------------------------------------------------------------- */
double orc_adaptive_eps(double eps, int64_t cV, int64_t cVp, int64_t k, int64_t kp, int32_t d) {
  double ratio = (1.0 + eps) * (double)kp * (double)cV / ((double)k * (double)cVp);
  return pow(ratio, 1.0 / (double)d) - 1.0;
}

/* Alg. 2: the subgraph induced by the vertices v with part[v] == b.  Phase  */
/* 1 counts n', w' and m' (CSR entries); phase 2 numbers the members by a     */
/* prefix sum of the indicator; phase 3 counts each member's neighbours in   */
/* the block, prefix-sums them into the row pointer and copies the edges in  */
/* adjacency order.  M[v] is v's id in the subgraph (-1 outside).  The       */
/* output arrays hold n' + 1, m', m' and n' entries.  Returns n'.            */
int32_t orc_build_subgraph(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                           const int32_t *vw, const int32_t *part, int32_t b, int64_t *xadj_s,
                           int32_t *adj_s, int32_t *adjw_s, int32_t *vw_s, int32_t *M, int64_t *out_m,
                           int64_t *out_w) {
  /* phase 1 */
  int32_t ns = 0;
  int64_t ws = 0, ms = 0;
  for (int32_t v = 0; v < n; v++)
    if (part[v] == b) { ns++; ws += vw[v]; }
  for (int32_t v = 0; v < n; v++)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++)
      if (part[v] == b && part[adj[e]] == b) ms++;
  /* phase 2: exclusive prefix sum of the indicator */
  int32_t run = 0;
  for (int32_t v = 0; v < n; v++) {
    if (part[v] == b) M[v] = run++;
    else M[v] = -1;
  }
  /* phase 3 */
  int64_t *D = (int64_t *)calloc((size_t)ns + 1, sizeof(int64_t));
  for (int32_t v = 0; v < n; v++) {
    if (part[v] != b) continue;
    int64_t d = 0;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) d += part[adj[e]] == b;
    D[M[v]] = d;
  }
  xadj_s[0] = 0;
  for (int32_t j = 0; j < ns; j++) xadj_s[j + 1] = xadj_s[j] + D[j];
  for (int32_t v = 0; v < n; v++) {
    if (part[v] != b) continue;
    int64_t i = xadj_s[M[v]];
    for (int64_t e = xadj[v]; e < xadj[v + 1]; e++) {
      if (part[adj[e]] != b) continue;
      adj_s[i] = M[adj[e]];
      adjw_s[i] = adjw[e];
      i++;
    }
    vw_s[M[v]] = vw[v];
  }
  free(D);
  if (out_m) *out_m = ms;
  if (out_w) *out_w = ws;
  return ns;
}

typedef struct {
  const int32_t *hier;
  double eps;
  int64_t cV, k;
  const orc_params *prm;
  int32_t *pi;
  orc_hm_stats *st;
} hm_job;

/* Alg. 3, one call: partition G' into a_i blocks with the multilevel        */
/* partitioner (the mapping pipeline on the one-level hierarchy a_i with      */
/* distance 1, whose J is twice the edge cut) under eps' (clamped to          */
/* [0, 1 - 10^-6]); at i = 1 the blocks are PEs, otherwise every block's      */
/* induced subgraph is partitioned one level down.  Block b at level i adds   */
/* b * a_1 ... a_{i-1} to the PE id (a_1 varies fastest).  orig maps the      */
/* subgraph's vertices to the input graph's.                                  */
static void hm_call(hm_job *J, int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                    const int32_t *vw, const int32_t *orig, int32_t i, int64_t base) {
  if (n == 0) return;
  int32_t a = J->hier[i - 1];
  int64_t kp = 1;
  for (int32_t j = 0; j < i; j++) kp *= J->hier[j];
  int64_t below = kp / a;
  int64_t cVp = 0;
  for (int32_t v = 0; v < n; v++) cVp += vw[v];
  double ep = orc_adaptive_eps(J->eps, J->cV, cVp, J->k, kp, i);
  if (ep < 0.0) ep = 0.0;
  if (ep > 0.999999) ep = 0.999999;
  int32_t one = 1;
  int32_t *part = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  orc_map_run(n, xadj, adj, adjw, vw, &a, &one, 1, ep, J->prm, part, NULL);
  if (J->st) {
    J->st->calls[i - 1]++;
    if (J->st->calls[i - 1] == 1) J->st->first_eps[i - 1] = ep;
  }
  if (i == 1) {
    for (int32_t v = 0; v < n; v++) J->pi[orig[v]] = (int32_t)(base + part[v]);
    free(part);
    return;
  }
  int64_t m = xadj[n];
  int64_t *xs = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t *as = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t *ws = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t *vs = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *M = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *os = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  for (int32_t b = 0; b < a; b++) {
    int32_t ns = orc_build_subgraph(n, xadj, adj, adjw, vw, part, b, xs, as, ws, vs, M, NULL, NULL);
    for (int32_t v = 0; v < n; v++)
      if (M[v] >= 0) os[M[v]] = orig[v];
    hm_call(J, ns, xs, as, ws, vs, os, i - 1, base + (int64_t)b * below);
  }
  free(xs); free(as); free(ws); free(vs); free(M); free(os); free(part);
}

int64_t orc_hm_run(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *adjw,
                   const int32_t *vw, const int32_t *hier, const int32_t *dist, int32_t levels,
                   double eps, const orc_params *prm, int32_t *pi, orc_hm_stats *stats) {
  hm_job J;
  orc_params part = *prm; /* the partitioner starts from breadth-first chunks */
  part.initial = 0;
  J.hier = hier;
  J.eps = eps;
  J.cV = 0;
  for (int32_t v = 0; v < n; v++) J.cV += vw[v];
  J.k = orc_num_pes(hier, levels);
  J.prm = &part;
  J.pi = pi;
  J.st = stats;
  if (stats) memset(stats, 0, sizeof(*stats));
  int32_t *orig = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  for (int32_t v = 0; v < n; v++) orig[v] = v;
  hm_call(&J, n, xadj, adj, adjw, vw, orig, levels, 0);
  free(orig);
  int64_t maxw = 0;
  return orc_objective(n, xadj, adj, adjw, vw, hier, dist, levels, pi, NULL, &maxw);
}
