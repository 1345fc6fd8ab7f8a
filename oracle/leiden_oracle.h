/*
 * leiden_oracle.h -- sequential CPU oracle for the Static, Naive-dynamic (ND),
 * Delta-screening (DS) and Dynamic Frontier (DF) Leiden of arXiv 2405.11658
 * ("A Starting Point for Dynamic Community Detection with Leiden Algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA library.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * load it; the product path never calls it.  It shares no code, header,
 * helper or constant table with the CUDA path.
 *
 * Conventions (all sizes in elements, all arrays owned by the caller):
 *   - graph: symmetric CSR, off[n+1] (int64), idx[off[n]] (int32),
 *     w[off[n]] (int64, > 0).  A self-loop (i,i,w) is stored once and adds w
 *     to K_i and to 2m (Sec. 3 definitions of K_i and m).
 *   - every integer quantity is exact: K, Sigma and 2m in int64, the scaled
 *     delta-modularity S (Eq. 2 times 2m^2 q) in __int128.
 *   - resolution gamma = p/q with q = 2^20 before reduction; p/q must be exact.
 *   - membership arrays hold community IDs in [0, n).
 *
 * Parity status: every function below is pinned by tests in tests/ that do
 * not call back into this file (closed forms, brute force, invariants).
 */
#ifndef LEIDEN_ORACLE_H
#define LEIDEN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SCHED_DET = 0, ORC_SCHED_GS = 1 };
enum { ORC_MODE_STATIC = 0, ORC_MODE_ND = 1, ORC_MODE_DS = 2, ORC_MODE_DF = 3 };

typedef struct {
  double gamma;                 /* resolution; Eq. 1/2 at gamma = 1 */
  double tol;                   /* initial iteration tolerance tau (Sec. 4.7: 0.01) */
  double tol_drop;              /* tau divisor per pass (Sec. 4.7: 10) */
  int32_t max_iters;            /* MAX_ITERATIONS (Sec. 4.7: 20) */
  int32_t max_passes;           /* MAX_PASSES (not stated; default 10) */
  int32_t sched;                /* ORC_SCHED_DET or ORC_SCHED_GS */
  int32_t det_subsets;          /* DET colour classes, power of two, 1..256 */
  int32_t refine_all_first_pass;/* Full Refine variant (Sec. 4.2) */
} orc_opts;

#define ORC_MAX_PASSES 64
typedef struct {
  int32_t passes;                   /* passes started */
  int32_t iters[ORC_MAX_PASSES];    /* l_i returned by leidenMove per pass */
  int64_t nv[ORC_MAX_PASSES];       /* |V'| at the start of each pass */
  int64_t nnz[ORC_MAX_PASSES];      /* CSR entries of G' at each pass */
  int64_t moves[ORC_MAX_PASSES];    /* local-move migrations per pass */
  int64_t refine_moves[ORC_MAX_PASSES];
  int64_t ncomm[ORC_MAX_PASSES];    /* communities after renumber, or -1 */
  double t_pass[ORC_MAX_PASSES];    /* seconds per pass */
  int64_t affected0;                /* vertices affected at the start of pass 0 */
  int64_t changed0;                 /* communities flagged changed before refine, pass 0 */
} orc_stats;

/* gamma -> p/q with q = 2^20, reduced by gcd; 0 if exact, -1 otherwise. */
int orc_gamma_ratio(double gamma, int64_t *p, int64_t *q);

/* 2m = total CSR weight. */
int64_t orc_two_m(int64_t n, const int64_t *off, const int64_t *w);

/* Eq. 1 at resolution gamma; also returns the exact numerator
 * q*2m*sum(sigma_c) - p*sum(Sigma_c^2) as two int64 words (lo, hi). */
double orc_modularity(int64_t n, const int64_t *off, const int32_t *idx,
                      const int64_t *w, const int32_t *C, double gamma,
                      int64_t *num_lo, int64_t *num_hi);

/* Scaled delta-modularity S of moving i from C[i] to c (Eq. 2 times 2m^2 q),
 * recomputed from scratch from C; out[0] = low word, out[1] = high word. */
void orc_move_score(int64_t n, const int64_t *off, const int32_t *idx,
                    const int64_t *w, const int32_t *C, int32_t i, int32_t c,
                    int64_t p, int64_t q, int64_t *out);

/* DET colour class of vertex i for S classes. */
int32_t orc_det_class(int64_t i, int32_t S);

/* Alg. leidenlm: local-moving phase.  Updates C, Sigma, changed, processed in
 * place; returns l_i (iterations performed, 1..max_iters).  in_range == NULL
 * means every vertex is in the affected range. */
int32_t orc_local_move(int64_t n, const int64_t *off, const int32_t *idx,
                       const int64_t *w, int32_t *C, const int64_t *K,
                       int64_t *Sigma, uint8_t *changed, uint8_t *processed,
                       const uint8_t *in_range, int32_t dynamic, int64_t p,
                       int64_t q, int64_t two_m, double tau, int32_t max_iters,
                       int32_t sched, int32_t S, int64_t *moves_out);

/* Alg. leidensr: relabel every community by its smallest member vertex. */
void orc_subset_renumber(int64_t n, int32_t *C, int64_t *Sigma, uint8_t *changed);

/* breakChangedCommunities of Alg. leiden. */
void orc_break_changed(int64_t n, int32_t *C, const int64_t *K, int64_t *Sigma,
                       const uint8_t *changed);

/* Alg. leidenre: one refinement sweep inside the bounds CB; returns moves. */
int64_t orc_refine(int64_t n, const int64_t *off, const int32_t *idx,
                   const int64_t *w, const int32_t *CB, int32_t *C,
                   const int64_t *K, int64_t *Sigma, const uint8_t *changed,
                   int64_t p, int64_t q, int64_t two_m, int32_t sched, int32_t S);

/* Dense renumbering of C in increasing order of old ID; returns |Gamma|. */
int64_t orc_renumber(int64_t n, int32_t *C);

/* Alg. leidenag: super-vertex graph of the dense membership C (nc communities).
 * off2[nc+1]; idx2/w2 need room for off[n] entries; rows sorted by target.
 * Returns nnz of the super-vertex graph. */
int64_t orc_aggregate(int64_t n, const int64_t *off, const int32_t *idx,
                      const int64_t *w, const int32_t *C, int64_t nc,
                      int64_t *off2, int32_t *idx2, int64_t *w2);

/* Alg. update on undirected pairs (each pair once, applied in both directions). */
void orc_update_weights(int64_t n, const int32_t *Cprev, int64_t *K, int64_t *Sigma,
                        int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *dw,
                        int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw);

/* changedCommunities of Alg. leiden (dynamic branch). */
void orc_changed_communities(int64_t n, const int32_t *Cprev, uint8_t *changed,
                             int64_t nd, const int32_t *ds, const int32_t *dd,
                             int64_t ni, const int32_t *is, const int32_t *id);

/* Initial affected vertices of Alg. frontier (DF). */
void orc_mark_df(int64_t n, const int32_t *Cprev, uint8_t *affected,
                 int64_t nd, const int32_t *ds, const int32_t *dd,
                 int64_t ni, const int32_t *is, const int32_t *id);

/* Affected vertices of Alg. delta (DS) on G^t, with K^t, Sigma^t. */
void orc_mark_ds(int64_t n, const int64_t *off, const int32_t *idx,
                 const int32_t *Cprev, const int64_t *K, const int64_t *Sigma,
                 int64_t p, int64_t q, int64_t two_m, uint8_t *affected,
                 int64_t nd, const int32_t *ds, const int32_t *dd,
                 int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw);

/* Alg. leiden: the dynamic-supporting driver.  affected == NULL: every vertex
 * starts unprocessed; changed == NULL: every community is changed.  Writes the
 * refined top-level membership (not canonicalised) to Cout. */
int orc_leiden(int64_t n, const int64_t *off, const int32_t *idx, const int64_t *w,
               const int32_t *Cprev, const int64_t *K, const int64_t *Sigma,
               const uint8_t *affected, int32_t range_is_affected,
               const uint8_t *changed, int32_t dynamic, const orc_opts *o,
               int32_t *Cout, orc_stats *st);

/* Canonical labels: community of the smallest member first, dense. */
int64_t orc_canonical(int64_t n, int32_t *C);

/* Static Leiden from singletons; canonical membership and Q. */
int orc_static(int64_t n, const int64_t *off, const int32_t *idx, const int64_t *w,
               const orc_opts *o, int32_t *Cout, double *q_out, orc_stats *st);

/* ND / DS / DF update (Alg. naive / delta / frontier) on G^t with the batch
 * that produced it.  Kprev/Sprev may be NULL (then K^t, Sigma^t are recomputed
 * from G^t and Cprev).  Outputs canonical C^t, K^t and Sigma^t indexed by the
 * canonical labels of C^t. */
int orc_update(int64_t n, const int64_t *off, const int32_t *idx, const int64_t *w,
               const int32_t *Cprev, const int64_t *Kprev, const int64_t *Sprev,
               int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *dw,
               int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw,
               int32_t mode, const orc_opts *o, int32_t *Cout, int64_t *Kout,
               int64_t *Sout, double *q_out, orc_stats *st);

#ifdef __cplusplus
}
#endif
#endif
