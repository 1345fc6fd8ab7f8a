/*
 * leiden_oracle.c -- plain sequential restatement of the Leiden variants of
 * arXiv 2405.11658.  TEST INFRASTRUCTURE ONLY: only tests/, the smoke check
 * and the benchmark's CPU-baseline leg may load this library.
 *
 * Each function cites the passage it follows.  Algorithms are named by their
 * LaTeX labels in the paper (Alg. leiden, leidenlm, leidensr, leidenre,
 * leidenag, update, naive, delta, frontier); equations by number (Eq. 1 is
 * modularity, Eq. 2 is delta-modularity).
 *
 * Where the paper is silent or ambiguous this file takes one reading and says
 * so at the spot ("reading:").  The full list is kept with the design notes.
 *
 * Data structures are deliberately simple: the per-vertex hashtable is a dense
 * array indexed by community ID plus a list of touched keys, the same
 * "collision-free" table the paper describes (Sec. 4.7), used by one thread.
 */
#define _POSIX_C_SOURCE 199309L
#include "leiden_oracle.h"

#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef __int128 i128;

static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void *xcalloc(size_t count, size_t size) {
  void *p = calloc(count ? count : 1, size);
  if (!p) abort();
  return p;
}

static void split128(i128 x, int64_t *lo, int64_t *hi) {
  *lo = (int64_t)(uint64_t)((unsigned __int128)x);
  *hi = (int64_t)(x >> 64);
}

/* ------------------------------------------------------------------------ */
/* Resolution: gamma = p / q exactly, q = 2^20 before reduction.             */
/* ------------------------------------------------------------------------ */
static int64_t gcd64(int64_t a, int64_t b) {
  while (b) { int64_t t = a % b; a = b; b = t; }
  return a;
}

int orc_gamma_ratio(double gamma, int64_t *p, int64_t *q) {
  const double Q = 1048576.0; /* 2^20 */
  double scaled = gamma * Q;
  if (!(gamma > 0.0) || scaled > 9.0e15) return -1;
  int64_t pp = (int64_t)scaled;
  if ((double)pp != scaled) return -1;
  int64_t qq = 1048576;
  int64_t g = gcd64(pp, qq);
  *p = pp / g;
  *q = qq / g;
  return 0;
}

int64_t orc_two_m(int64_t n, const int64_t *off, const int64_t *w) {
  int64_t s = 0;
  for (int64_t e = 0; e < off[n]; e++) s += w[e];
  return s;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: Q = sum_c [ sigma_c / 2m - gamma (Sigma_c / 2m)^2 ].               */
/* sigma_c sums w_ij over ordered pairs (CSR entries) with both ends in c;   */
/* Sigma_c sums K_i over i in c (Sec. 3 definitions).                        */
/* ------------------------------------------------------------------------ */
double orc_modularity(int64_t n, const int64_t *off, const int32_t *idx,
                      const int64_t *w, const int32_t *C, double gamma,
                      int64_t *num_lo, int64_t *num_hi) {
  int64_t p = 1, q = 1;
  if (orc_gamma_ratio(gamma, &p, &q) != 0) { p = 1; q = 1; }
  int64_t two_m = 0, sigma_in = 0;
  int64_t *Sig = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) {
    for (int64_t e = off[i]; e < off[i + 1]; e++) {
      two_m += w[e];
      Sig[C[i]] += w[e];
      if (C[idx[e]] == C[i]) sigma_in += w[e];
    }
  }
  i128 sq = 0;
  for (int64_t c = 0; c < n; c++) sq += (i128)Sig[c] * Sig[c];
  free(Sig);
  i128 num = (i128)q * two_m * sigma_in - (i128)p * sq;
  if (num_lo && num_hi) split128(num, num_lo, num_hi);
  if (two_m == 0) return 0.0;
  double den = (double)two_m * (double)two_m * (double)q;
  return (double)num / den;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2 scaled by 2m^2 q:                                                   */
/*   S = 2m q (K_{i->c} - K_{i->d}) - p K_i (K_i + Sigma_c - Sigma_d)        */
/* ------------------------------------------------------------------------ */
static i128 score(int64_t two_m, int64_t p, int64_t q, int64_t Kic, int64_t Kid,
                  int64_t Ki, int64_t Sc, int64_t Sd) {
  return (i128)two_m * q * (Kic - Kid) - (i128)p * Ki * (Ki + Sc - Sd);
}

void orc_move_score(int64_t n, const int64_t *off, const int32_t *idx,
                    const int64_t *w, const int32_t *C, int32_t i, int32_t c,
                    int64_t p, int64_t q, int64_t *out) {
  int64_t two_m = 0, Ki = 0, Kic = 0, Kid = 0, Sc = 0, Sd = 0;
  int32_t d = C[i];
  for (int64_t u = 0; u < n; u++) {
    int64_t ku = 0;
    for (int64_t e = off[u]; e < off[u + 1]; e++) ku += w[e];
    two_m += ku;
    if (C[u] == c) Sc += ku;
    if (C[u] == d) Sd += ku;
  }
  for (int64_t e = off[i]; e < off[i + 1]; e++) {
    Ki += w[e];
    if (idx[e] == i) continue; /* scanCommunities with self = false */
    if (C[idx[e]] == c) Kic += w[e];
    if (C[idx[e]] == d) Kid += w[e];
  }
  split128(score(two_m, p, q, Kic, Kid, Ki, Sc, Sd), &out[0], &out[1]);
}

/* ------------------------------------------------------------------------ */
/* DET schedule (our definition; the paper's run is asynchronous, Sec. 4.7): */
/* S colour classes by a multiplicative hash of the vertex ID.               */
/* ------------------------------------------------------------------------ */
static int ilog2_pow2(int32_t S) {
  int k = 0;
  while ((1 << k) < S) k++;
  return k;
}

int32_t orc_det_class(int64_t i, int32_t S) {
  int k = ilog2_pow2(S);
  if (k == 0) return 0;
  uint32_t h = (uint32_t)i * 2654435761u;
  return (int32_t)(h >> (32 - k));
}

/* ------------------------------------------------------------------------ */
/* Dense-array hashtable (Sec. 4.7 "collision-free per-thread hashtable").   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t *val;   /* [n], zero when unused */
  uint8_t *used;  /* [n] */
  int32_t *keys;  /* touched keys */
  int64_t nkeys;
} table;

static void table_init(table *t, int64_t n) {
  t->val = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  t->used = (uint8_t *)xcalloc((size_t)n, 1);
  t->keys = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  t->nkeys = 0;
}
static void table_free(table *t) { free(t->val); free(t->used); free(t->keys); }
static void table_add(table *t, int32_t k, int64_t v) {
  if (!t->used[k]) { t->used[k] = 1; t->keys[t->nkeys++] = k; }
  t->val[k] += v;
}
static void table_clear(table *t) {
  for (int64_t a = 0; a < t->nkeys; a++) {
    t->val[t->keys[a]] = 0;
    t->used[t->keys[a]] = 0;
  }
  t->nkeys = 0;
}

/* scanCommunities (Alg. leidenlm) with self = false, and scanBounded
 * (Alg. leidenre) when CB != NULL. */
static void scan_row(table *t, const int64_t *off, const int32_t *idx,
                     const int64_t *w, const int32_t *C, const int32_t *CB,
                     int32_t i) {
  for (int64_t e = off[i]; e < off[i + 1]; e++) {
    int32_t j = idx[e];
    if (j == i) continue;
    if (CB && CB[j] != CB[i]) continue;
    table_add(t, C[j], w[e]);
  }
}

/* Best community among the keys of the table other than d.
 * reading: ties go to the smallest community ID (the paper is silent). */
static int best_move(const table *t, int32_t d, int64_t Ki, const int64_t *Sigma,
                     int64_t p, int64_t q, int64_t two_m, int32_t *cbest, i128 *Sbest) {
  int64_t Kid = t->used[d] ? t->val[d] : 0;
  int found = 0;
  for (int64_t a = 0; a < t->nkeys; a++) {
    int32_t c = t->keys[a];
    if (c == d) continue;
    i128 S = score(two_m, p, q, t->val[c], Kid, Ki, Sigma[c], Sigma[d]);
    if (!found || S > *Sbest || (S == *Sbest && c < *cbest)) {
      found = 1;
      *Sbest = S;
      *cbest = c;
    }
  }
  return found;
}

/* ------------------------------------------------------------------------ */
/* Alg. leidenlm -- local-moving phase.                                      */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t i, c; i128 S; } proposal;

static void apply_move(int32_t i, int32_t cstar, int64_t Ki, int32_t *C,
                       int64_t *Sigma, uint8_t *changed, uint8_t *processed,
                       const int64_t *off, const int32_t *idx, int32_t dynamic) {
  int32_t d = C[i];
  Sigma[d] -= Ki;
  Sigma[cstar] += Ki;
  C[i] = cstar;
  /* vertex pruning: a mover re-marks its neighbours (which is also DF's
   * onChange, Alg. frontier) */
  for (int64_t e = off[i]; e < off[i + 1]; e++) processed[idx[e]] = 0;
  if (dynamic) { changed[d] = 1; changed[cstar] = 1; }
}

int32_t orc_local_move(int64_t n, const int64_t *off, const int32_t *idx,
                       const int64_t *w, int32_t *C, const int64_t *K,
                       int64_t *Sigma, uint8_t *changed, uint8_t *processed,
                       const uint8_t *in_range, int32_t dynamic, int64_t p,
                       int64_t q, int64_t two_m, double tau, int32_t max_iters,
                       int32_t sched, int32_t S, int64_t *moves_out) {
  table t;
  table_init(&t, n);
  proposal *props = (proposal *)xcalloc((size_t)n, sizeof(proposal));
  /* denominator turning the integer sum back into delta-modularity:
   * sum(S) / (2 m^2 q) with 2 m^2 = (2m)^2 / 2 */
  double den = (double)two_m * (double)two_m * 0.5 * (double)q;
  int64_t moves = 0;
  int32_t li = 0;
  int32_t nsub = (sched == ORC_SCHED_DET) ? S : 1;
  while (li < max_iters) {
    i128 sumS = 0;
    for (int32_t s = 0; s < nsub; s++) {
      int64_t np = 0;
      for (int64_t i = 0; i < n; i++) {
        if (sched == ORC_SCHED_DET && orc_det_class(i, S) != s) continue;
        if (processed[i]) continue;
        processed[i] = 1;                         /* prune */
        if (in_range && !in_range[i]) continue;   /* inAffectedRange */
        scan_row(&t, off, idx, w, C, NULL, (int32_t)i);
        int32_t cstar = -1;
        i128 Sbest = 0;
        int found = best_move(&t, C[i], K[i], Sigma, p, q, two_m, &cstar, &Sbest);
        table_clear(&t);
        /* reading: move only to a strictly better community (S > 0) */
        if (!found || Sbest <= 0) continue;
        if (sched == ORC_SCHED_GS) {
          apply_move((int32_t)i, cstar, K[i], C, Sigma, changed, processed,
                     off, idx, dynamic);
          sumS += Sbest;
          moves++;
        } else {
          props[np].i = (int32_t)i;
          props[np].c = cstar;
          props[np].S = Sbest;
          np++;
        }
      }
      /* DET: every move of the sub-sweep was chosen against the same
       * snapshot; apply them together now. */
      for (int64_t a = 0; a < np; a++) {
        apply_move(props[a].i, props[a].c, K[props[a].i], C, Sigma, changed,
                   processed, off, idx, dynamic);
        sumS += props[a].S;
        moves++;
      }
    }
    li++;
    /* locally converged when the iteration's total delta-modularity <= tau */
    if (two_m == 0 || (double)sumS / den <= tau) break;
  }
  free(props);
  table_free(&t);
  if (moves_out) *moves_out = moves;
  return li;
}

/* ------------------------------------------------------------------------ */
/* Alg. leidensr -- renumber each community by a member vertex.              */
/* reading: the member chosen is the smallest vertex ID ("any vertex").      */
/* ------------------------------------------------------------------------ */
void orc_subset_renumber(int64_t n, int32_t *C, int64_t *Sigma, uint8_t *changed) {
  int32_t *rep = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  int64_t *S2 = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  uint8_t *ch2 = (uint8_t *)xcalloc((size_t)n, 1);
  for (int64_t c = 0; c < n; c++) rep[c] = -1;
  for (int64_t i = 0; i < n; i++)
    if (rep[C[i]] < 0) rep[C[i]] = (int32_t)i; /* increasing i: the minimum */
  for (int64_t c = 0; c < n; c++) {
    if (rep[c] < 0) continue;
    S2[rep[c]] = Sigma[c];
    ch2[rep[c]] = changed[c];
  }
  for (int64_t i = 0; i < n; i++) C[i] = rep[C[i]];
  memcpy(Sigma, S2, (size_t)n * sizeof(int64_t));
  memcpy(changed, ch2, (size_t)n);
  free(rep); free(S2); free(ch2);
}

/* breakChangedCommunities (Alg. leiden). */
void orc_break_changed(int64_t n, int32_t *C, const int64_t *K, int64_t *Sigma,
                       const uint8_t *changed) {
  /* decide membership first: the flag is indexed by the community before the
   * break, which other vertices of the same community must still see */
  uint8_t *brk = (uint8_t *)xcalloc((size_t)n, 1);
  for (int64_t i = 0; i < n; i++) brk[i] = changed[C[i]];
  for (int64_t i = 0; i < n; i++) {
    if (!brk[i]) continue;
    C[i] = (int32_t)i;
    Sigma[i] = K[i];
  }
  free(brk);
}

/* ------------------------------------------------------------------------ */
/* Alg. leidenre -- refinement (constrained merge), one sweep.               */
/* reading: the changed-flag test uses the flag of i's bound, changed[CB[i]] */
/* (after the break C'[i] = i, so the literal index cannot be meant).        */
/* DET: a proposal i -> c* is accepted iff c* made no proposal in the same   */
/* sub-sweep; this replaces the compare-and-swap race deterministically.     */
/* ------------------------------------------------------------------------ */
int64_t orc_refine(int64_t n, const int64_t *off, const int32_t *idx,
                   const int64_t *w, const int32_t *CB, int32_t *C,
                   const int64_t *K, int64_t *Sigma, const uint8_t *changed,
                   int64_t p, int64_t q, int64_t two_m, int32_t sched, int32_t S) {
  table t;
  table_init(&t, n);
  proposal *props = (proposal *)xcalloc((size_t)n, sizeof(proposal));
  uint8_t *proposed = (uint8_t *)xcalloc((size_t)n, 1);
  int64_t moves = 0;
  int32_t nsub = (sched == ORC_SCHED_DET) ? S : 1;
  for (int32_t s = 0; s < nsub; s++) {
    int64_t np = 0;
    for (int64_t i = 0; i < n; i++) {
      if (sched == ORC_SCHED_DET && orc_det_class(i, S) != s) continue;
      if (!changed[CB[i]]) continue;
      int32_t c = C[i];
      if (Sigma[c] != K[i]) continue; /* not isolated any more */
      scan_row(&t, off, idx, w, C, CB, (int32_t)i);
      int32_t cstar = -1;
      i128 Sbest = 0;
      int found = best_move(&t, c, K[i], Sigma, p, q, two_m, &cstar, &Sbest);
      table_clear(&t);
      if (!found || Sbest <= 0) continue;
      if (C[cstar] != cstar) continue; /* the target's own vertex has left */
      if (sched == ORC_SCHED_GS) {
        /* atomicCAS(Sigma[c], K[i], 0) succeeds: sequential execution */
        Sigma[c] = 0;
        Sigma[cstar] += K[i];
        C[i] = cstar;
        moves++;
      } else {
        props[np].i = (int32_t)i;
        props[np].c = cstar;
        props[np].S = Sbest;
        np++;
        proposed[i] = 1;
      }
    }
    for (int64_t a = 0; a < np; a++) {
      int32_t i = props[a].i, cstar = props[a].c;
      if (proposed[cstar]) continue;
      Sigma[C[i]] -= K[i];
      Sigma[cstar] += K[i];
      C[i] = cstar;
      moves++;
    }
    for (int64_t a = 0; a < np; a++) proposed[props[a].i] = 0;
  }
  free(proposed);
  free(props);
  table_free(&t);
  return moves;
}

/* ------------------------------------------------------------------------ */
/* "Renumber communities in C'" (Alg. leiden): dense IDs in increasing order */
/* of the old ID.                                                            */
/* ------------------------------------------------------------------------ */
int64_t orc_renumber(int64_t n, int32_t *C) {
  int32_t *id = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  uint8_t *exists = (uint8_t *)xcalloc((size_t)n, 1);
  for (int64_t i = 0; i < n; i++) exists[C[i]] = 1;
  int64_t k = 0;
  for (int64_t c = 0; c < n; c++) id[c] = exists[c] ? (int32_t)k++ : -1;
  for (int64_t i = 0; i < n; i++) C[i] = id[C[i]];
  free(id); free(exists);
  return k;
}

/* ------------------------------------------------------------------------ */
/* Alg. leidenag -- aggregation into a super-vertex graph.                   */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

int64_t orc_aggregate(int64_t n, const int64_t *off, const int32_t *idx,
                      const int64_t *w, const int32_t *C, int64_t nc,
                      int64_t *off2, int32_t *idx2, int64_t *w2) {
  /* community-vertex CSR: countCommunityVertices + exclusive scan + placement */
  int64_t *coff = (int64_t *)xcalloc((size_t)nc + 1, sizeof(int64_t));
  int32_t *cv = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
  int64_t *cur = (int64_t *)xcalloc((size_t)nc, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) coff[C[i] + 1]++;
  for (int64_t c = 0; c < nc; c++) coff[c + 1] += coff[c];
  for (int64_t i = 0; i < n; i++) cv[coff[C[i]] + cur[C[i]]++] = (int32_t)i;
  /* per community: scanCommunities with self = true over every member row */
  table t;
  table_init(&t, nc > 0 ? nc : 1);
  int64_t m2 = 0;
  off2[0] = 0;
  for (int64_t c = 0; c < nc; c++) {
    for (int64_t a = coff[c]; a < coff[c + 1]; a++) {
      int32_t i = cv[a];
      for (int64_t e = off[i]; e < off[i + 1]; e++) table_add(&t, C[idx[e]], w[e]);
    }
    qsort(t.keys, (size_t)t.nkeys, sizeof(int32_t), cmp_i32);
    for (int64_t a = 0; a < t.nkeys; a++) {
      idx2[m2] = t.keys[a];
      w2[m2] = t.val[t.keys[a]];
      m2++;
    }
    off2[c + 1] = m2;
    table_clear(&t);
  }
  table_free(&t);
  free(coff); free(cv); free(cur);
  return m2;
}

/* ------------------------------------------------------------------------ */
/* Alg. update -- K^t and Sigma^t from K^{t-1}, Sigma^{t-1} and the batch.   */
/* Every undirected pair (u,v,w) stands for the directed entries (u,v,w) and */
/* (v,u,w) (Sec. 5.1.4: every update carries its reverse edge).              */
/* ------------------------------------------------------------------------ */
void orc_update_weights(int64_t n, const int32_t *Cprev, int64_t *K, int64_t *Sigma,
                        int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *dw,
                        int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw) {
  (void)n;
  for (int64_t a = 0; a < nd; a++) {
    int32_t ends[2] = {ds[a], dd[a]};
    for (int k = 0; k < 2; k++) {
      int32_t i = ends[k];
      K[i] -= dw[a];
      Sigma[Cprev[i]] -= dw[a];
    }
  }
  for (int64_t a = 0; a < ni; a++) {
    int32_t ends[2] = {is[a], id[a]};
    for (int k = 0; k < 2; k++) {
      int32_t i = ends[k];
      K[i] += iw[a];
      Sigma[Cprev[i]] += iw[a];
    }
  }
}

/* changedCommunities (Alg. leiden), reading: the flag written is that of the
 * shared community, changed[C^{t-1}[i]] ("mark the community as changed",
 * Sec. 4.3). */
void orc_changed_communities(int64_t n, const int32_t *Cprev, uint8_t *changed,
                             int64_t nd, const int32_t *ds, const int32_t *dd,
                             int64_t ni, const int32_t *is, const int32_t *id) {
  (void)n;
  for (int64_t a = 0; a < nd; a++)
    if (Cprev[ds[a]] == Cprev[dd[a]]) changed[Cprev[ds[a]]] = 1;
  for (int64_t a = 0; a < ni; a++)
    if (Cprev[is[a]] == Cprev[id[a]]) changed[Cprev[is[a]]] = 1;
}

/* Alg. frontier: deletions inside a community and insertions across
 * communities mark their source; both directions are in the batch. */
void orc_mark_df(int64_t n, const int32_t *Cprev, uint8_t *affected,
                 int64_t nd, const int32_t *ds, const int32_t *dd,
                 int64_t ni, const int32_t *is, const int32_t *id) {
  (void)n;
  for (int64_t a = 0; a < nd; a++)
    if (Cprev[ds[a]] == Cprev[dd[a]]) { affected[ds[a]] = 1; affected[dd[a]] = 1; }
  for (int64_t a = 0; a < ni; a++)
    if (Cprev[is[a]] != Cprev[id[a]]) { affected[is[a]] = 1; affected[id[a]] = 1; }
}

/* Alg. delta (DS).  reading: for each source i of cross-community insertions,
 * H[c] sums the inserted weight towards c != C[i]; c* maximises Eq. 2 (scaled)
 * with K_{i->c} = H[c], K_{i->d} = 0 and K^t, Sigma^t; ties to the smallest
 * c.  A source whose insertions all stay inside its community marks nothing. */
void orc_mark_ds(int64_t n, const int64_t *off, const int32_t *idx,
                 const int32_t *Cprev, const int64_t *K, const int64_t *Sigma,
                 int64_t p, int64_t q, int64_t two_m, uint8_t *affected,
                 int64_t nd, const int32_t *ds, const int32_t *dd,
                 int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw) {
  uint8_t *dE = (uint8_t *)xcalloc((size_t)n, 1);
  uint8_t *dC = (uint8_t *)xcalloc((size_t)n, 1);
  /* deletions inside one community: i, its neighbours and its community */
  for (int64_t a = 0; a < nd; a++) {
    int32_t u = ds[a], v = dd[a];
    if (Cprev[u] != Cprev[v]) continue;
    affected[u] = 1; dE[u] = 1; dC[Cprev[v]] = 1;
    affected[v] = 1; dE[v] = 1; dC[Cprev[u]] = 1;
  }
  /* insertions: group the directed entries by source (the batch "sorted by
   * source", Appendix A.2) with a counting sort */
  int64_t ne = 2 * ni;
  int64_t *soff = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  int64_t *cur = (int64_t *)xcalloc((size_t)n, sizeof(int64_t));
  int32_t *sdst = (int32_t *)xcalloc((size_t)(ne ? ne : 1), sizeof(int32_t));
  int32_t *swt = (int32_t *)xcalloc((size_t)(ne ? ne : 1), sizeof(int32_t));
  for (int64_t a = 0; a < ni; a++) { soff[is[a] + 1]++; soff[id[a] + 1]++; }
  for (int64_t i = 0; i < n; i++) soff[i + 1] += soff[i];
  for (int64_t a = 0; a < ni; a++) {
    int64_t x = soff[is[a]] + cur[is[a]]++;
    sdst[x] = id[a]; swt[x] = iw[a];
    x = soff[id[a]] + cur[id[a]]++;
    sdst[x] = is[a]; swt[x] = iw[a];
  }
  table t;
  table_init(&t, n);
  for (int64_t i = 0; i < n; i++) {
    if (soff[i + 1] == soff[i]) continue;
    for (int64_t x = soff[i]; x < soff[i + 1]; x++)
      if (Cprev[sdst[x]] != Cprev[i]) table_add(&t, Cprev[sdst[x]], swt[x]);
    if (t.nkeys > 0) {
      int32_t d = Cprev[i];
      int32_t cstar = -1;
      i128 Sbest = 0;
      for (int64_t a = 0; a < t.nkeys; a++) {
        int32_t c = t.keys[a];
        i128 S = score(two_m, p, q, t.val[c], 0, K[i], Sigma[c], Sigma[d]);
        if (cstar < 0 || S > Sbest || (S == Sbest && c < cstar)) { Sbest = S; cstar = c; }
      }
      affected[i] = 1; dE[i] = 1; dC[cstar] = 1;
    }
    table_clear(&t);
  }
  table_free(&t);
  /* expand: neighbours of dE vertices, members of dC communities */
  for (int64_t i = 0; i < n; i++) {
    if (dE[i])
      for (int64_t e = off[i]; e < off[i + 1]; e++) affected[idx[e]] = 1;
    if (dC[Cprev[i]]) affected[i] = 1;
  }
  free(dE); free(dC); free(soff); free(cur); free(sdst); free(swt);
}

/* ------------------------------------------------------------------------ */
/* Alg. leiden -- passes of local-move, subset renumber, break, refine,      */
/* renumber, dendrogram lookup and aggregation.                              */
/* ------------------------------------------------------------------------ */
int orc_leiden(int64_t n, const int64_t *off, const int32_t *idx, const int64_t *w,
               const int32_t *Cprev, const int64_t *K, const int64_t *Sigma,
               const uint8_t *affected, int32_t range_is_affected,
               const uint8_t *changed, int32_t dynamic, const orc_opts *o,
               int32_t *Cout, orc_stats *st) {
  int64_t p, q;
  if (orc_gamma_ratio(o->gamma, &p, &q) != 0) return -1;
  int32_t S = o->det_subsets > 0 ? o->det_subsets : 1;
  if (st) memset(st, 0, sizeof(*st));
  int64_t two_m = orc_two_m(n, off, w);

  /* mark affected vertices as unprocessed */
  uint8_t *processed = (uint8_t *)xcalloc((size_t)(n ? n : 1), 1);
  int64_t naff = 0;
  for (int64_t i = 0; i < n; i++) {
    processed[i] = affected ? !affected[i] : 0;
    naff += !processed[i];
  }
  if (st) st->affected0 = naff;

  /* initialisation */
  for (int64_t i = 0; i < n; i++) Cout[i] = (int32_t)i;     /* C */
  int64_t nv = n;
  const int64_t *goff = off;                                 /* G' */
  const int32_t *gidx = idx;
  const int64_t *gw = w;
  int64_t *own_off = NULL, *own_w = NULL;
  int32_t *own_idx = NULL;
  int32_t *Cp = (int32_t *)xcalloc((size_t)(n ? n : 1), sizeof(int32_t));   /* C' */
  int32_t *CB = (int32_t *)xcalloc((size_t)(n ? n : 1), sizeof(int32_t));   /* C'_B */
  int64_t *Kp = (int64_t *)xcalloc((size_t)(n ? n : 1), sizeof(int64_t));   /* K' */
  int64_t *Sp = (int64_t *)xcalloc((size_t)(n ? n : 1), sizeof(int64_t));   /* Sigma' */
  uint8_t *ch = (uint8_t *)xcalloc((size_t)(n ? n : 1), 1);                 /* Delta C' */
  memcpy(Cp, Cprev, (size_t)n * sizeof(int32_t));
  memcpy(Kp, K, (size_t)n * sizeof(int64_t));
  memcpy(Sp, Sigma, (size_t)n * sizeof(int64_t));
  for (int64_t c = 0; c < n; c++)
    ch[c] = (changed && !o->refine_all_first_pass) ? changed[c] : 1;

  double tau = o->tol;
  int32_t lp;
  for (lp = 0; lp < o->max_passes; lp++) {
    double t0 = now_s();
    if (st && lp < ORC_MAX_PASSES) {
      st->passes = lp + 1;
      st->nv[lp] = nv;
      st->nnz[lp] = goff[nv];
      st->ncomm[lp] = -1;
    }
    const uint8_t *rng = (lp == 0 && range_is_affected) ? affected : NULL;
    int64_t moves = 0;
    int32_t li = orc_local_move(nv, goff, gidx, gw, Cp, Kp, Sp, ch, processed,
                                rng, dynamic && lp == 0, p, q, two_m, tau,
                                o->max_iters, o->sched, S, &moves);
    if (st && lp == 0) {
      int64_t nch = 0;
      for (int64_t c = 0; c < nv; c++) nch += ch[c] != 0;
      st->changed0 = nch;
    }
    orc_subset_renumber(nv, Cp, Sp, ch);
    memcpy(CB, Cp, (size_t)nv * sizeof(int32_t));
    orc_break_changed(nv, Cp, Kp, Sp, ch);
    int64_t rmoves = orc_refine(nv, goff, gidx, gw, CB, Cp, Kp, Sp, ch, p, q,
                                two_m, o->sched, S);
    if (st && lp < ORC_MAX_PASSES) {
      st->iters[lp] = li;
      st->moves[lp] = moves;
      st->refine_moves[lp] = rmoves;
    }
    if (lp > 0 && li <= 1) {                 /* globally converged */
      if (st && lp < ORC_MAX_PASSES) st->t_pass[lp] = now_s() - t0;
      break;
    }
    int64_t nc = orc_renumber(nv, Cp);
    if (st && lp < ORC_MAX_PASSES) st->ncomm[lp] = nc;
    /* reading: aggregation that would not shrink the graph cannot make
     * progress (aggregation tolerance 1, Sec. 5.1.2): stop */
    if (nc == nv) {
      if (st && lp < ORC_MAX_PASSES) st->t_pass[lp] = now_s() - t0;
      break;
    }
    for (int64_t v = 0; v < n; v++) Cout[v] = Cp[Cout[v]];  /* dendrogram lookup */
    int64_t *noff = (int64_t *)xcalloc((size_t)nc + 1, sizeof(int64_t));
    int32_t *nidx = (int32_t *)xcalloc((size_t)(goff[nv] ? goff[nv] : 1), sizeof(int32_t));
    int64_t *nw = (int64_t *)xcalloc((size_t)(goff[nv] ? goff[nv] : 1), sizeof(int64_t));
    orc_aggregate(nv, goff, gidx, gw, Cp, nc, noff, nidx, nw);
    free(own_off); free(own_idx); free(own_w);
    own_off = noff; own_idx = nidx; own_w = nw;
    goff = noff; gidx = nidx; gw = nw;
    nv = nc;
    for (int64_t c = 0; c < nv; c++) {          /* K' = Sigma' = row sums */
      int64_t s = 0;
      for (int64_t e = goff[c]; e < goff[c + 1]; e++) s += gw[e];
      Kp[c] = s;
      Sp[c] = s;
      processed[c] = 0;                          /* all unprocessed */
      Cp[c] = (int32_t)c;                        /* refine-based labels */
      ch[c] = 1;                                 /* refine all next pass */
    }
    tau /= o->tol_drop;
    if (st && lp < ORC_MAX_PASSES) st->t_pass[lp] = now_s() - t0;
  }
  for (int64_t v = 0; v < n; v++) Cout[v] = Cp[Cout[v]];    /* final lookup */
  free(own_off); free(own_idx); free(own_w);
  free(Cp); free(CB); free(Kp); free(Sp); free(ch); free(processed);
  return 0;
}

int64_t orc_canonical(int64_t n, int32_t *C) {
  int32_t *lab = (int32_t *)xcalloc((size_t)(n ? n : 1), sizeof(int32_t));
  for (int64_t c = 0; c < n; c++) lab[c] = -1;
  int64_t k = 0;
  for (int64_t v = 0; v < n; v++)
    if (lab[C[v]] < 0) lab[C[v]] = (int32_t)k++;
  for (int64_t v = 0; v < n; v++) C[v] = lab[C[v]];
  free(lab);
  return k;
}

static void row_sums(int64_t n, const int64_t *off, const int64_t *w, int64_t *K) {
  for (int64_t i = 0; i < n; i++) {
    int64_t s = 0;
    for (int64_t e = off[i]; e < off[i + 1]; e++) s += w[e];
    K[i] = s;
  }
}

int orc_static(int64_t n, const int64_t *off, const int32_t *idx, const int64_t *w,
               const orc_opts *o, int32_t *Cout, double *q_out, orc_stats *st) {
  int32_t *C0 = (int32_t *)xcalloc((size_t)(n ? n : 1), sizeof(int32_t));
  int64_t *K = (int64_t *)xcalloc((size_t)(n ? n : 1), sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) C0[i] = (int32_t)i;
  row_sums(n, off, w, K);
  /* Static: all vertices affected, every community changed, Sigma = K */
  int rc = orc_leiden(n, off, idx, w, C0, K, K, NULL, 0, NULL, 0, o, Cout, st);
  free(C0); free(K);
  if (rc) return rc;
  orc_canonical(n, Cout);
  if (q_out) *q_out = orc_modularity(n, off, idx, w, Cout, o->gamma, NULL, NULL);
  return 0;
}

int orc_update(int64_t n, const int64_t *off, const int32_t *idx, const int64_t *w,
               const int32_t *Cprev, const int64_t *Kprev, const int64_t *Sprev,
               int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *dw,
               int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw,
               int32_t mode, const orc_opts *o, int32_t *Cout, int64_t *Kout,
               int64_t *Sout, double *q_out, orc_stats *st) {
  int64_t p, q;
  if (orc_gamma_ratio(o->gamma, &p, &q) != 0) return -1;
  size_t nn = (size_t)(n ? n : 1);
  int64_t *K = (int64_t *)xcalloc(nn, sizeof(int64_t));
  int64_t *Sg = (int64_t *)xcalloc(nn, sizeof(int64_t));
  if (Kprev && Sprev) {
    memcpy(K, Kprev, (size_t)n * sizeof(int64_t));
    memcpy(Sg, Sprev, (size_t)n * sizeof(int64_t));
    orc_update_weights(n, Cprev, K, Sg, nd, ds, dd, dw, ni, is, id, iw);
  } else {
    row_sums(n, off, w, K);
    for (int64_t i = 0; i < n; i++) Sg[Cprev[i]] += K[i];
  }
  int64_t two_m = orc_two_m(n, off, w);
  uint8_t *ch = (uint8_t *)xcalloc(nn, 1);
  orc_changed_communities(n, Cprev, ch, nd, ds, dd, ni, is, id);
  uint8_t *aff = NULL;
  int32_t range_is_aff = 0;
  if (mode == ORC_MODE_DF) {
    aff = (uint8_t *)xcalloc(nn, 1);
    orc_mark_df(n, Cprev, aff, nd, ds, dd, ni, is, id);
  } else if (mode == ORC_MODE_DS) {
    aff = (uint8_t *)xcalloc(nn, 1);
    orc_mark_ds(n, off, idx, Cprev, K, Sg, p, q, two_m, aff, nd, ds, dd, ni, is, id, iw);
    range_is_aff = 1;
  } else if (mode != ORC_MODE_ND) {
    free(K); free(Sg); free(ch);
    return -1;
  }
  int rc = orc_leiden(n, off, idx, w, Cprev, K, Sg, aff, range_is_aff, ch, 1, o, Cout, st);
  free(aff); free(ch);
  if (rc) { free(K); free(Sg); return rc; }
  orc_canonical(n, Cout);
  /* reading: Sigma^t is returned for the new membership C^t so the next
   * update starts from consistent auxiliary information */
  if (Kout) memcpy(Kout, K, (size_t)n * sizeof(int64_t));
  if (Sout) {
    memset(Sout, 0, (size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) Sout[Cout[i]] += K[i];
  }
  if (q_out) *q_out = orc_modularity(n, off, idx, w, Cout, o->gamma, NULL, NULL);
  free(K); free(Sg);
  return 0;
}
