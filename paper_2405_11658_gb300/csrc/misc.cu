// misc.cu -- the small phases of Alg. leiden and the dynamic front-ends:
// weighted degrees, subset renumbering (Alg. leidensr), breakChangedCommunities,
// dense renumbering, dendrogram lookup, canonical labels, modularity terms
// (Eq. 1), updateWeights (Alg. update), changedCommunities and DF marking
// (Alg. frontier).
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace lk {

static inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// K_i = sum of the row (self-loop included once), warp per vertex.
template <typename WT>
__global__ void row_sums_k(GraphView<WT> g, int64_t *K) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < g.n; i += nw) {
    int64_t s = 0;
    for (int64_t e = g.off[i] + lane; e < g.off[i + 1]; e += 32) s += (int64_t)g.w[e];
    for (int o = 16; o; o >>= 1) s += shfl_xor_i64(s, o);
    if (lane == 0) K[i] = s;
  }
}
template <typename WT>
void launch_row_sums(GraphView<WT> g, int64_t *K, cudaStream_t s) {
  if (g.n <= 0) return;
  LK_COUNTED row_sums_k<WT><<<grid_for(g.n * 32, 256, 152 * 64), 256, 0, s>>>(g, K);
}
template void launch_row_sums<int32_t>(GraphView<int32_t>, int64_t *, cudaStream_t);
template void launch_row_sums<int64_t>(GraphView<int64_t>, int64_t *, cudaStream_t);

__global__ void iota_k(int32_t *a, int64_t n) { GRID_STRIDE(i, n) a[i] = (int32_t)i; }
void launch_iota(int32_t *a, int64_t n, cudaStream_t s) {
  if (n > 0) LK_COUNTED iota_k<<<grid_for(n, 256), 256, 0, s>>>(a, n);
}
__global__ void fill_u8_k(uint8_t *a, uint8_t v, int64_t n) { GRID_STRIDE(i, n) a[i] = v; }
void launch_fill_u8(uint8_t *a, uint8_t v, int64_t n, cudaStream_t s) {
  if (n > 0) cudaMemsetAsync(a, v, (size_t)n, s);
}
void launch_copy_i64(int64_t *dst, const int64_t *src, int64_t n, cudaStream_t s) {
  if (n > 0) cudaMemcpyAsync(dst, src, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
}
__global__ void invert_u8_k(uint8_t *d, const uint8_t *a, int64_t n) { GRID_STRIDE(i, n) d[i] = a[i] ? 0 : 1; }
// After an ASYNC refinement: the totals of communities whose own vertex left
// hold the departure marker; those communities are empty.
__global__ void clear_left_k(int64_t *Sig, int64_t n) { GRID_STRIDE(i, n) if (Sig[i] < 0) Sig[i] = 0; }
void launch_clear_left(int64_t *Sig, int64_t n, cudaStream_t s) {
  if (n > 0) LK_COUNTED clear_left_k<<<grid_for(n, 256), 256, 0, s>>>(Sig, n);
}
void launch_invert_u8(uint8_t *dst, const uint8_t *src, int64_t n, cudaStream_t s) {
  if (n > 0) LK_COUNTED invert_u8_k<<<grid_for(n, 256), 256, 0, s>>>(dst, src, n);
}

__global__ void sum_i64_k(const int64_t *a, int64_t n, u64 *out) {
  __shared__ int64_t sbuf[32];
  int64_t s = 0;
  GRID_STRIDE(i, n) s += a[i];
  s = block_sum_i64(s, sbuf);
  if (threadIdx.x == 0 && s) atomicAdd(out, (u64)s);
}
void launch_sum_i64(const int64_t *a, int64_t n, u64 *out, cudaStream_t s) {
  if (n > 0) LK_COUNTED sum_i64_k<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(a, n, out);
}

// ---------------------------------------------------------------------------
// Alg. leidensr: relabel each community by a member vertex (the smallest).
// ---------------------------------------------------------------------------
__global__ void sr_init_k(int64_t n, int32_t *rep, int64_t *Sig2, uint8_t *ch2) {
  GRID_STRIDE(c, n) { rep[c] = INT_MAX; Sig2[c] = 0; ch2[c] = 0; }
}
// The minima only fall: a member that reads a representative already below
// its own ID cannot lower it, and skips the atomic (a large community's
// members would otherwise queue on one address).
__global__ void sr_min_k(int64_t n, const int32_t *C, int32_t *rep) {
  GRID_STRIDE(i, n) {
    const int32_t c = C[i];
    if (rep[c] > (int32_t)i) atomicMin(&rep[c], (int32_t)i);
  }
}
__global__ void sr_move_k(int64_t n, const int32_t *rep, const int64_t *Sig, int64_t *Sig2,
                          const uint8_t *ch, uint8_t *ch2) {
  GRID_STRIDE(c, n) {
    const int32_t r = rep[c];
    if (r == INT_MAX) continue;
    Sig2[r] = Sig[c];
    ch2[r] = ch[c];
  }
}
__global__ void sr_relabel_k(int64_t n, int32_t *C, const int32_t *rep) {
  GRID_STRIDE(i, n) C[i] = rep[C[i]];
}
void launch_subset_renumber(int64_t n, int32_t *C, const int64_t *Sig, int64_t *Sig2,
                            const uint8_t *ch, uint8_t *ch2, int32_t *rep, cudaStream_t s) {
  if (n <= 0) return;
  const unsigned g = grid_for(n, 256);
  LK_COUNTED sr_init_k<<<g, 256, 0, s>>>(n, rep, Sig2, ch2);
  LK_COUNTED sr_min_k<<<g, 256, 0, s>>>(n, C, rep);
  LK_COUNTED sr_move_k<<<g, 256, 0, s>>>(n, rep, Sig, Sig2, ch, ch2);
  LK_COUNTED sr_relabel_k<<<g, 256, 0, s>>>(n, C, rep);
}

// breakChangedCommunities: every vertex of a changed community becomes its
// own community.  Thread i reads only C'[i] and the flags, writes C'[i] and
// Sigma'[i]; no other thread reads Sigma' here.
__global__ void break_k(int64_t n, int32_t *C, const int64_t *K, int64_t *Sig, const uint8_t *ch) {
  GRID_STRIDE(i, n) {
    if (!ch[C[i]]) continue;
    C[i] = (int32_t)i;
    Sig[i] = K[i];
  }
}
void launch_break(int64_t n, int32_t *C, const int64_t *K, int64_t *Sig, const uint8_t *ch,
                  cudaStream_t s) {
  if (n > 0) LK_COUNTED break_k<<<grid_for(n, 256), 256, 0, s>>>(n, C, K, Sig, ch);
}

// Dense renumbering in increasing order of the old ID (flag + exclusive scan).
__global__ void flag_k(int64_t n, const int32_t *C, uint8_t *ex) {
  GRID_STRIDE(i, n) {
    const int32_t c = C[i];
    if (!ex[c]) ex[c] = 1;   // most members find the flag set already: spare the store
  }
}
__global__ void relabel_scan_k(int64_t n, int32_t *C, const int64_t *scanned) {
  GRID_STRIDE(i, n) C[i] = (int32_t)scanned[C[i]];
}
__global__ void store_total_k(const int64_t *scanned, int64_t n, u64 *dst) { *dst = (u64)scanned[n]; }
void launch_renumber(int64_t n, int32_t *C, uint8_t *exists, int64_t *scanned, int64_t *tmp,
                     u64 *ctr, cudaStream_t s) {
  cudaMemsetAsync(exists, 0, (size_t)(n > 0 ? n : 1), s);
  if (n > 0) LK_COUNTED flag_k<<<grid_for(n, 256), 256, 0, s>>>(n, C, exists);
  exclusive_scan<uint8_t>(exists, scanned, n, tmp, s);
  if (n > 0) LK_COUNTED relabel_scan_k<<<grid_for(n, 256), 256, 0, s>>>(n, C, scanned);
  LK_COUNTED store_total_k<<<1, 1, 0, s>>>(scanned, n, &ctr[CTR_NCOMM]);
}

// Dendrogram lookup C[v] <- C'[C[v]].
__global__ void lookup_k(int64_t n, int32_t *Ctop, const int32_t *Cp) {
  GRID_STRIDE(v, n) Ctop[v] = Cp[Ctop[v]];
}
void launch_lookup(int64_t n, int32_t *Ctop, const int32_t *Cp, cudaStream_t s) {
  if (n > 0) LK_COUNTED lookup_k<<<grid_for(n, 256), 256, 0, s>>>(n, Ctop, Cp);
}

// Canonical labels: communities numbered by their smallest member vertex.
__global__ void canon_init_k(int64_t n, int32_t *minv, uint8_t *flag) {
  GRID_STRIDE(i, n) { minv[i] = INT_MAX; flag[i] = 0; }
}
__global__ void canon_min_k(int64_t n, const int32_t *C, int32_t *minv) {
  GRID_STRIDE(v, n) {
    const int32_t c = C[v];
    if (minv[c] > (int32_t)v) atomicMin(&minv[c], (int32_t)v);   // as in sr_min_k
  }
}
__global__ void canon_flag_k(int64_t n, const int32_t *minv, uint8_t *flag) {
  GRID_STRIDE(c, n) if (minv[c] != INT_MAX) flag[minv[c]] = 1;
}
__global__ void canon_out_k(int64_t n, const int32_t *C, const int32_t *minv, const int64_t *scanned,
                            int32_t *out) {
  GRID_STRIDE(v, n) out[v] = (int32_t)scanned[minv[C[v]]];
}
void launch_canonical(int64_t n, const int32_t *C, int32_t *out, int32_t *minv, uint8_t *flag,
                      int64_t *scanned, int64_t *tmp, cudaStream_t s) {
  if (n <= 0) return;
  const unsigned g = grid_for(n, 256);
  LK_COUNTED canon_init_k<<<g, 256, 0, s>>>(n, minv, flag);
  LK_COUNTED canon_min_k<<<g, 256, 0, s>>>(n, C, minv);
  LK_COUNTED canon_flag_k<<<g, 256, 0, s>>>(n, minv, flag);
  exclusive_scan<uint8_t>(flag, scanned, n, tmp, s);
  LK_COUNTED canon_out_k<<<g, 256, 0, s>>>(n, C, minv, scanned, out);
}

// ---------------------------------------------------------------------------
// Eq. 1 terms: acc[0] = sum of internal weight (sum_c sigma_c), acc[1..2] =
// sum_c Sigma_c^2 (i128), acc[3] = 2m.
//
// Every index is tested before it is used -- the row bounds against [0, nnz],
// the labels and column IDs against [0, n) -- so a malformed input can never
// make these kernels read or write outside the arrays, whatever the caller
// has or has not validated: an offending row or entry is skipped and sets
// 512 in *err.  A kernel that finds *err already set (an earlier check on
// the same stream failed) does nothing.
// ---------------------------------------------------------------------------
template <typename WT>
__global__ void mod_rows_k(GraphView<WT> g, int64_t nnz, const int32_t *C, int64_t *Sig, u64 *acc,
                           u64 *err) {
  __shared__ int64_t sbuf[32];
  __shared__ int s_skip;
  // one reading for the whole block, so no thread skips the barriers below
  // while another waits at them
  if (threadIdx.x == 0) s_skip = *(volatile u64 *)err != 0;
  __syncthreads();
  if (s_skip) return;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t inside = 0, total = 0;
  bool bad = false;
  for (int64_t i = w0; i < g.n; i += nw) {
    const int64_t e0 = g.off[i], e1 = g.off[i + 1];
    const int32_t ci = C[i];
    if (e0 < 0 || e1 < e0 || e1 > nnz || ci < 0 || (int64_t)ci >= g.n) { bad = true; continue; }
    int64_t k = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int64_t w = (int64_t)g.w[e];
      const int32_t j = g.idx[e];
      if (j < 0 || (int64_t)j >= g.n) { bad = true; continue; }
      k += w;
      if (C[j] == ci) inside += w;
    }
    for (int o = 16; o; o >>= 1) k += shfl_xor_i64(k, o);
    if (lane == 0 && k) { atomic_add_i64(&Sig[ci], k); total += k; }
  }
  if (bad) atomicOr(err, 512ull);
  inside = block_sum_i64(inside, sbuf);
  total = block_sum_i64(total, sbuf);
  if (threadIdx.x == 0) {
    if (inside) atomicAdd(&acc[0], (u64)inside);
    if (total) atomicAdd(&acc[3], (u64)total);
  }
}
__global__ void mod_sq_k(int64_t n, const int64_t *Sig, u64 *acc) {
  __shared__ i128 sbuf[32];
  i128 s = 0;
  GRID_STRIDE(c, n) s += (i128)Sig[c] * Sig[c];
  s = block_sum_i128(s, sbuf);
  if (threadIdx.x == 0 && s != 0) atomic_add_i128(&acc[1], s);
}
template <typename WT>
void launch_modularity_terms(GraphView<WT> g, int64_t nnz, const int32_t *C, int64_t *Sig_tmp, u64 *acc,
                             u64 *err, cudaStream_t s) {
  cudaMemsetAsync(acc, 0, 4 * sizeof(u64), s);
  if (g.n <= 0) return;
  cudaMemsetAsync(Sig_tmp, 0, (size_t)g.n * sizeof(int64_t), s);
  LK_COUNTED mod_rows_k<WT><<<grid_for(g.n * 32, 256, 152 * 32), 256, 0, s>>>(g, nnz, C, Sig_tmp, acc, err);
  LK_COUNTED mod_sq_k<<<grid_for(g.n, 256, 152 * 8), 256, 0, s>>>(g.n, Sig_tmp, acc);
}
template void launch_modularity_terms<int32_t>(GraphView<int32_t>, int64_t, const int32_t *, int64_t *, u64 *,
                                               u64 *, cudaStream_t);
template void launch_modularity_terms<int64_t>(GraphView<int64_t>, int64_t, const int32_t *, int64_t *, u64 *,
                                               u64 *, cudaStream_t);

// Sigma[c] = sum of K over members of c (Sigma zeroed first).
__global__ void sigma_from_k(int64_t n, const int32_t *C, const int64_t *K, int64_t *Sig) {
  GRID_STRIDE(i, n) if (K[i]) atomic_add_i64(&Sig[C[i]], K[i]);
}
void launch_sigma_from(int64_t n, const int32_t *C, const int64_t *K, int64_t *Sig, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(Sig, 0, (size_t)n * sizeof(int64_t), s);
  LK_COUNTED sigma_from_k<<<grid_for(n, 256), 256, 0, s>>>(n, C, K, Sig);
}

// ---------------------------------------------------------------------------
// Batch handling.  Every undirected pair (u, v, w) stands for (u,v,w) and
// (v,u,w).
// ---------------------------------------------------------------------------
// Alg. update: K[i] += sign*w, Sigma[C^{t-1}[i]] += sign*w for both ends.
__global__ void update_weights_k(int64_t cnt, const int32_t *src, const int32_t *dst, const int32_t *w,
                                 int sign, const int32_t *Cprev, int64_t *K, int64_t *Sig) {
  GRID_STRIDE(k, cnt) {
    const int64_t x = sign * (int64_t)w[k];
    const int32_t u = src[k], v = dst[k];
    atomic_add_i64(&K[u], x);
    atomic_add_i64(&Sig[Cprev[u]], x);
    atomic_add_i64(&K[v], x);
    atomic_add_i64(&Sig[Cprev[v]], x);
  }
}
void launch_update_weights(int64_t count, const int32_t *src, const int32_t *dst, const int32_t *w,
                           int sign, const int32_t *Cprev, int64_t *K, int64_t *Sig, cudaStream_t s) {
  if (count > 0) LK_COUNTED update_weights_k<<<grid_for(count, 256), 256, 0, s>>>(count, src, dst, w, sign, Cprev, K, Sig);
}

// changedCommunities (reading: the flag of the shared community).
__global__ void changed_k(int64_t cnt, const int32_t *src, const int32_t *dst, const int32_t *Cprev,
                          uint8_t *changed) {
  GRID_STRIDE(k, cnt) {
    const int32_t cu = Cprev[src[k]];
    if (cu == Cprev[dst[k]]) changed[cu] = 1;
  }
}
void launch_changed_communities(int64_t count, const int32_t *src, const int32_t *dst,
                                const int32_t *Cprev, uint8_t *changed, cudaStream_t s) {
  if (count > 0) LK_COUNTED changed_k<<<grid_for(count, 256), 256, 0, s>>>(count, src, dst, Cprev, changed);
}

// Alg. frontier: deletions inside a community (same = 1) and insertions across
// communities (same = 0) mark both ends.
__global__ void mark_df_k(int64_t cnt, const int32_t *src, const int32_t *dst, const int32_t *Cprev,
                          int same, uint8_t *aff) {
  GRID_STRIDE(k, cnt) {
    const int32_t u = src[k], v = dst[k];
    if ((Cprev[u] == Cprev[v]) == (same != 0)) { aff[u] = 1; aff[v] = 1; }
  }
}
void launch_mark_df(int64_t count, const int32_t *src, const int32_t *dst, const int32_t *Cprev,
                    int same, uint8_t *affected, cudaStream_t s) {
  if (count > 0) LK_COUNTED mark_df_k<<<grid_for(count, 256), 256, 0, s>>>(count, src, dst, Cprev, same, affected);
}

// A CSR is well formed: off[0] = 0, off[n] = nnz, offsets non-decreasing,
// column IDs in [0, n), weights > 0.  Sets *err on violation.
__global__ void check_graph_rows_k(int64_t n, int64_t nnz, const int64_t *off, u64 *err) {
  GRID_STRIDE(i, n) {
    const int64_t a = off[i], b = off[i + 1];
    if (a > b || a < 0 || b > nnz) atomicOr(err, 128ull);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n] != nnz)) atomicOr(err, 128ull);
}
__global__ void check_graph_entries_k(int64_t n, int64_t nnz, const int32_t *idx, const int32_t *w, u64 *err) {
  GRID_STRIDE(e, nnz) if (idx[e] < 0 || idx[e] >= n || w[e] <= 0) atomicOr(err, 256ull);
}
void launch_check_graph(int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx, const int32_t *w,
                        u64 *err, cudaStream_t s) {
  LK_COUNTED check_graph_rows_k<<<grid_for(n > 0 ? n : 1, 256), 256, 0, s>>>(n, nnz, off, err);
  if (nnz > 0) LK_COUNTED check_graph_entries_k<<<grid_for(nnz, 256, 152 * 32), 256, 0, s>>>(n, nnz, idx, w, err);
}

// Labels in [0, hi); sets *err on violation.
__global__ void check_range_k(const int32_t *a, int64_t n, int64_t hi, u64 *err) {
  GRID_STRIDE(i, n) if (a[i] < 0 || a[i] >= hi) atomicOr(err, 32ull);
}
void launch_check_range(const int32_t *a, int64_t n, int64_t hi, u64 *err, cudaStream_t s) {
  if (n > 0) LK_COUNTED check_range_k<<<grid_for(n, 256), 256, 0, s>>>(a, n, hi, err);
}

// IDs in [0, n), no self-loops, positive weights; sets *err on violation.
__global__ void check_ids_k(int64_t cnt, const int32_t *src, const int32_t *dst, const int32_t *w,
                            int64_t n, u64 *err) {
  GRID_STRIDE(k, cnt) {
    const int32_t u = src[k], v = dst[k];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v || (w && w[k] <= 0)) atomicOr(err, 1ull);
  }
}
void launch_check_ids(int64_t count, const int32_t *src, const int32_t *dst, const int32_t *w,
                      int64_t n, u64 *err, cudaStream_t s) {
  if (count > 0) LK_COUNTED check_ids_k<<<grid_for(count, 256), 256, 0, s>>>(count, src, dst, w, n, err);
}

}  // namespace lk
