// dyn.cu -- Delta-screening marking (Alg. delta) and batch application
// G^{t-1} -> G^t (Sec. 3.5) on sm_103a.
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace lk {

static inline unsigned gridd(int64_t n, int threads, int64_t cap = 1 << 20) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}
#define DSTRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// Alg. delta.
// ---------------------------------------------------------------------------
// Deletions inside one community: mark the vertex, its neighbours (dE) and the
// community (dC), for both directions.
__global__ void ds_del_k(int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *Cprev,
                         uint8_t *aff, uint8_t *dE, uint8_t *dC) {
  DSTRIDE(k, nd) {
    const int32_t u = ds[k], v = dd[k];
    const int32_t c = Cprev[u];
    if (c != Cprev[v]) continue;
    aff[u] = 1; dE[u] = 1;
    aff[v] = 1; dE[v] = 1;
    dC[c] = 1;
  }
}
// Directed insertion entries grouped by source (counting sort).
__global__ void ds_cnt_k(int64_t ni, const int32_t *is, const int32_t *id, int64_t *cnt) {
  DSTRIDE(k, ni) {
    atomicAdd((u64 *)&cnt[is[k]], 1ull);
    atomicAdd((u64 *)&cnt[id[k]], 1ull);
  }
}
__global__ void ds_place_k(int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw,
                           const int64_t *soff, int64_t *cur, int32_t *sdst, int32_t *swt) {
  DSTRIDE(k, ni) {
    const int32_t u = is[k], v = id[k], w = iw[k];
    int64_t x = soff[u] + (int64_t)atomicAdd((u64 *)&cur[u], 1ull);
    sdst[x] = v; swt[x] = w;
    x = soff[v] + (int64_t)atomicAdd((u64 *)&cur[v], 1ull);
    sdst[x] = u; swt[x] = w;
  }
}
// One thread per source with insertions.  H[c] = inserted weight towards each
// community c != C^{t-1}[i]; c* maximises Eq. 2 (scaled) with K_{i->c} = H[c],
// K_{i->d} = 0, K^t and Sigma^t; ties go to the smallest c (reading).
__global__ void ds_best_k(int64_t n, const int64_t *soff, const int32_t *sdst, const int32_t *swt,
                          const int32_t *Cprev, const int64_t *K, const int64_t *Sig, int64_t A,
                          int64_t p, uint8_t *aff, uint8_t *dE, uint8_t *dC) {
  DSTRIDE(i, n) {
    const int64_t b = soff[i], e = soff[i + 1];
    if (b == e) continue;
    const int32_t d = Cprev[i];
    const int64_t Ki = K[i];
    int32_t best = INT_MAX;
    i128 bS = 0;
    for (int64_t x = b; x < e; x++) {
      const int32_t c = Cprev[sdst[x]];
      if (c == d) continue;
      bool seen = false;
      for (int64_t y = b; y < x; y++)
        if (Cprev[sdst[y]] == c) { seen = true; break; }
      if (seen) continue;
      int64_t h = 0;
      for (int64_t y = x; y < e; y++)
        if (Cprev[sdst[y]] == c) h += swt[y];
      const i128 S = (i128)A * h - (i128)p * Ki * (Ki + Sig[c] - Sig[d]);
      if (best == INT_MAX || S > bS || (S == bS && c < best)) { bS = S; best = c; }
    }
    if (best != INT_MAX) {
      aff[i] = 1;
      dE[i] = 1;
      dC[best] = 1;
    }
  }
}
// Expansion: neighbours of dE vertices and members of dC communities.
__global__ void ds_expand_k(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *Cprev,
                            const uint8_t *dE, const uint8_t *dC, uint8_t *aff) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i0 = w0 * 32; i0 < n; i0 += nw * 32) {
    const int64_t i = i0 + lane;
    bool e = false;
    if (i < n) {
      if (dC[Cprev[i]]) aff[i] = 1;
      e = dE[i] != 0;
    }
    unsigned m = __ballot_sync(FULL_MASK, e);
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
      const int64_t v = i0 + l;
      for (int64_t x = off[v] + lane; x < off[v + 1]; x += 32) aff[idx[x]] = 1;
    }
  }
}

void launch_mark_ds(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *Cprev,
                    const int64_t *K, const int64_t *Sig, int64_t A, int64_t p,
                    int64_t nd, const int32_t *ds, const int32_t *dd,
                    int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw,
                    uint8_t *affected, const DsWork &wk, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(wk.dE, 0, (size_t)n, s);
  cudaMemsetAsync(wk.dC, 0, (size_t)n, s);
  if (nd > 0) LK_COUNTED ds_del_k<<<gridd(nd, 256), 256, 0, s>>>(nd, ds, dd, Cprev, affected, wk.dE, wk.dC);
  if (ni > 0) {
    cudaMemsetAsync(wk.cnt, 0, (size_t)(n + 1) * sizeof(int64_t), s);
    cudaMemsetAsync(wk.cur, 0, (size_t)(n + 1) * sizeof(int64_t), s);
    LK_COUNTED ds_cnt_k<<<gridd(ni, 256), 256, 0, s>>>(ni, is, id, wk.cnt);
    exclusive_scan<int64_t>(wk.cnt, wk.soff, n, wk.scan_tmp, s);
    LK_COUNTED ds_place_k<<<gridd(ni, 256), 256, 0, s>>>(ni, is, id, iw, wk.soff, wk.cur, wk.sdst, wk.swt);
    LK_COUNTED ds_best_k<<<gridd(n, 256), 256, 0, s>>>(n, wk.soff, wk.sdst, wk.swt, Cprev, K, Sig, A, p, affected,
                                            wk.dE, wk.dC);
  }
  LK_COUNTED ds_expand_k<<<gridd(n, 256, 152 * 32), 256, 0, s>>>(n, off, idx, Cprev, wk.dE, wk.dC, affected);
}

// ---------------------------------------------------------------------------
// Batch application.  Rows of G^{t-1} are sorted; deletions remove an
// existing edge of the given weight; insertions of a pair already present (or
// repeated) add their weights; output rows are sorted.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t row_find(const int32_t *idx, int64_t b, int64_t e, int32_t v) {
  while (b < e) {
    const int64_t mid = (b + e) >> 1;
    if (idx[mid] < v) b = mid + 1; else e = mid;
  }
  return b;
}

// Sets the byte and returns its previous value.
__device__ __forceinline__ uint8_t atomic_set_byte(uint8_t *p) {
  const uintptr_t a = (uintptr_t)p;
  unsigned int *word = (unsigned int *)(a & ~(uintptr_t)3);
  const unsigned int sh = (unsigned int)(a & 3) * 8;
  const unsigned int old = atomicOr(word, 1u << sh);
  return (uint8_t)((old >> sh) & 0xffu);
}

__global__ void ba_deg_k(int64_t n, const int64_t *off, int64_t *newdeg) {
  DSTRIDE(u, n) newdeg[u] = off[u + 1] - off[u];
}
__global__ void ba_del_k(int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *dw,
                         const int64_t *off, const int32_t *idx, const int32_t *w, uint8_t *delmark,
                         int64_t *newdeg, u64 *err) {
  DSTRIDE(k, nd) {
    for (int dir = 0; dir < 2; dir++) {
      const int32_t u = dir ? dd[k] : ds[k], v = dir ? ds[k] : dd[k];
      const int64_t e = row_find(idx, off[u], off[u + 1], v);
      if (e >= off[u + 1] || idx[e] != v || w[e] != dw[k]) { atomicOr(err, 2ull); continue; }
      if (atomic_set_byte(&delmark[e])) { atomicOr(err, 4ull); continue; }
      atomicAdd((u64 *)&newdeg[u], (u64)-1ll);
    }
  }
}
// One thread per row with insertions: sort the row's new entries by target
// (insertion sort; rows get few of them), merge repeats, then count the output
// row length by merging with the surviving old entries.
__global__ void ba_ins_row_k(int64_t n, const int64_t *ioff, int32_t *idst, int32_t *iwt,
                             const int64_t *off, const int32_t *idx, const uint8_t *delmark,
                             int64_t *newdeg) {
  DSTRIDE(u, n) {
    const int64_t b = ioff[u], e = ioff[u + 1];
    if (b == e) continue;
    for (int64_t x = b + 1; x < e; x++) {
      const int32_t kv = idst[x], kw = iwt[x];
      int64_t y = x - 1;
      while (y >= b && idst[y] > kv) { idst[y + 1] = idst[y]; iwt[y + 1] = iwt[y]; y--; }
      idst[y + 1] = kv; iwt[y + 1] = kw;
    }
    // merge repeats into the first copy, mark the rest with -1
    for (int64_t x = b + 1; x < e; x++) {
      int64_t f = x - 1;
      while (f > b && idst[f] == -1) f--;
      if (idst[x] == idst[f]) { iwt[f] += iwt[x]; idst[x] = -1; }
    }
    int64_t len = 0;
    int64_t a = off[u];
    const int64_t a1 = off[u + 1];
    int64_t x = b;
    while (true) {
      while (x < e && idst[x] == -1) x++;
      while (a < a1 && delmark[a]) a++;
      if (x >= e && a >= a1) break;
      if (x >= e) { len++; a++; continue; }
      if (a >= a1) { len++; x++; continue; }
      if (idx[a] < idst[x]) { len++; a++; }
      else if (idx[a] > idst[x]) { len++; x++; }
      else { len++; a++; x++; }
    }
    newdeg[u] = len;
  }
}
// Warp per row: rows without insertions copy their surviving entries with a
// ballot compaction; rows with insertions are merged by lane 0.
__global__ void ba_write_k(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *w,
                           const uint8_t *delmark, const int64_t *ioff, const int32_t *idst,
                           const int32_t *iwt, const int64_t *off2, int32_t *idx2, int32_t *w2,
                           u64 *err) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = w0; u < n; u += nw) {
    const int64_t a0 = off[u], a1 = off[u + 1];
    // rows must be sorted (strictly: no duplicate entries)
    for (int64_t a = a0 + 1 + lane; a < a1; a += 32)
      if (idx[a - 1] >= idx[a]) atomicOr(err, 8ull);
    const int64_t b = ioff[u], e = ioff[u + 1];
    int64_t out = off2[u];
    if (b == e) {
      for (int64_t a = a0; a < a1; a += 32) {
        const int64_t x = a + lane;
        const bool keep = x < a1 && !delmark[x];
        const unsigned m = __ballot_sync(FULL_MASK, keep);
        if (keep) {
          const int64_t pos = out + __popc(m & ((1u << lane) - 1u));
          idx2[pos] = idx[x];
          w2[pos] = w[x];
        }
        out += __popc(m);
      }
      continue;
    }
    if (lane == 0) {
      int64_t a = a0, x = b;
      while (true) {
        while (x < e && idst[x] == -1) x++;
        while (a < a1 && delmark[a]) a++;
        if (x >= e && a >= a1) break;
        if (x >= e || (a < a1 && idx[a] < idst[x])) { idx2[out] = idx[a]; w2[out] = w[a]; a++; }
        else if (a >= a1 || idx[a] > idst[x]) { idx2[out] = idst[x]; w2[out] = iwt[x]; x++; }
        else { idx2[out] = idx[a]; w2[out] = w[a] + iwt[x]; a++; x++; }
        out++;
      }
    }
    __syncwarp();
  }
}

int apply_batch(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *w,
                int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *dw,
                int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw,
                int64_t *off_out, int32_t *idx_out, int32_t *w_out, int64_t cap_nnz,
                int64_t *nnz_out, const BatchWork &wk, cudaStream_t s) {
  cudaMemsetAsync(wk.err, 0, sizeof(u64), s);
  launch_check_ids(nd, ds, dd, dw, n, wk.err, s);
  launch_check_ids(ni, is, id, iw, n, wk.err, s);
  int64_t nnz = 0;
  cudaMemcpyAsync(&nnz, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  u64 herr = 0;
  cudaMemcpyAsync(&herr, wk.err, sizeof(u64), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
  if (herr) return LEIDEN_EINVAL;
  if (nnz > 0) cudaMemsetAsync(wk.delmark, 0, (size_t)nnz, s);
  if (n > 0) LK_COUNTED ba_deg_k<<<gridd(n, 256), 256, 0, s>>>(n, off, wk.newdeg);
  if (nd > 0) LK_COUNTED ba_del_k<<<gridd(nd, 256), 256, 0, s>>>(nd, ds, dd, dw, off, idx, w, wk.delmark, wk.newdeg, wk.err);
  cudaMemsetAsync(wk.cnt, 0, (size_t)(n + 1) * sizeof(int64_t), s);
  cudaMemsetAsync(wk.cur, 0, (size_t)(n + 1) * sizeof(int64_t), s);
  if (ni > 0) LK_COUNTED ds_cnt_k<<<gridd(ni, 256), 256, 0, s>>>(ni, is, id, wk.cnt);
  exclusive_scan<int64_t>(wk.cnt, wk.ioff, n, wk.scan_tmp, s);
  if (ni > 0) {
    LK_COUNTED ds_place_k<<<gridd(ni, 256), 256, 0, s>>>(ni, is, id, iw, wk.ioff, wk.cur, wk.idst, wk.iwt);
    LK_COUNTED ba_ins_row_k<<<gridd(n, 128), 128, 0, s>>>(n, wk.ioff, wk.idst, wk.iwt, off, idx, wk.delmark, wk.newdeg);
  }
  exclusive_scan<int64_t>(wk.newdeg, off_out, n, wk.scan_tmp, s);
  int64_t nnz2 = 0;
  cudaMemcpyAsync(&nnz2, off_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&herr, wk.err, sizeof(u64), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
  if (herr) return LEIDEN_EINVAL;
  if (nnz2 > cap_nnz) return LEIDEN_ENOMEM;
  if (n > 0)
    LK_COUNTED ba_write_k<<<gridd(n * 32, 256, 152 * 32), 256, 0, s>>>(n, off, idx, w, wk.delmark, wk.ioff, wk.idst, wk.iwt,
                                                             off_out, idx_out, w_out, wk.err);
  cudaMemcpyAsync(&herr, wk.err, sizeof(u64), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
  if (herr) return LEIDEN_EINVAL;
  *nnz_out = nnz2;
  return LEIDEN_OK;
}

}  // namespace lk
