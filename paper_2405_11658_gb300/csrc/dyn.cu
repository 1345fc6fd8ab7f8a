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
// repeated) add their weights; deletions apply before insertions; output rows
// are sorted.
//
// Only the rows the batch touches are merged.  Every directed update goes to
// its row's list (counting sort by row); one thread per touched row sorts its
// list, merges equal targets and classifies each target against the old row
// (removed, reweighted, new), which gives the row's new length; the untouched
// rows between two touched ones keep their entries in order, shifted by the
// same amount, so they are copied as runs of entries; one warp per touched row
// places its surviving old entries and new entries by rank.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t row_find(const int32_t *idx, int64_t b, int64_t e, int32_t v) {
  while (b < e) {
    const int64_t mid = (b + e) >> 1;
    if (idx[mid] < v) b = mid + 1; else e = mid;
  }
  return b;
}

enum { UPD_REMOVED = 1, UPD_REWEIGHT = 2, UPD_NEW = 3 };

__global__ void ba_deg_k(int64_t n, const int64_t *off, int64_t *newdeg) {
  DSTRIDE(u, n) newdeg[u] = off[u + 1] - off[u];
}
// Both directions of every update counted by row.
__global__ void ba_cnt_k(int64_t cnt_, const int32_t *s, const int32_t *d, int64_t *cnt) {
  DSTRIDE(k, cnt_) {
    atomicAdd((u64 *)&cnt[s[k]], 1ull);
    atomicAdd((u64 *)&cnt[d[k]], 1ull);
  }
}
// Places both directions of every update in its row's list: target and signed
// weight (deletions negative; weights were checked positive).
__global__ void ba_place_k(int64_t cnt_, const int32_t *s, const int32_t *d, const int32_t *w, int sign,
                           const int64_t *uoff, int64_t *cur, int32_t *ut, int32_t *uw) {
  DSTRIDE(k, cnt_) {
    const int32_t u = s[k], v = d[k], x = sign * w[k];
    int64_t p = uoff[u] + (int64_t)atomicAdd((u64 *)&cur[u], 1ull);
    ut[p] = v; uw[p] = x;
    p = uoff[v] + (int64_t)atomicAdd((u64 *)&cur[v], 1ull);
    ut[p] = u; uw[p] = x;
  }
}
__global__ void ba_touched_flag_k(int64_t n, const int64_t *cnt, uint8_t *tflag) {
  DSTRIDE(u, n) tflag[u] = cnt[u] > 0;
}
__global__ void ba_touched_list_k(int64_t n, const uint8_t *tflag, const int64_t *tpos, int32_t *trow) {
  DSTRIDE(u, n) if (tflag[u]) trow[tpos[u]] = (int32_t)u;
}
// One thread per touched row: sort the row's updates by target (insertion
// sort: a row gets few), merge equal targets, classify each against the old
// row and record the exclusive prefix counts of removed and new entries.
// Writes the compacted records to the front of the row's list, their count to
// nrec[u] and the new row length to newdeg[u].
__global__ void ba_row_k(int64_t T, const int32_t *trow, const int64_t *uoff, int32_t *ut, int32_t *uw,
                         uint8_t *uk, int32_t *Rp, int32_t *Np, int64_t *nrec, const int64_t *off,
                         const int32_t *idx, const int32_t *w, int64_t *newdeg, u64 *err) {
  DSTRIDE(t, T) {
    const int32_t u = trow[t];
    const int64_t b = uoff[u], e = uoff[u + 1];
    for (int64_t x = b + 1; x < e; x++) {
      const int32_t kv = ut[x], kw = uw[x];
      int64_t y = x - 1;
      while (y >= b && ut[y] > kv) { ut[y + 1] = ut[y]; uw[y + 1] = uw[y]; y--; }
      ut[y + 1] = kv; uw[y + 1] = kw;
    }
    const int64_t a0 = off[u], a1 = off[u + 1];
    int32_t R = 0, N = 0;
    int64_t q = b;
    for (int64_t x = b; x < e;) {
      const int32_t tgt = ut[x];
      int64_t dw = 0, iw = 0;
      int dels = 0;
      for (; x < e && ut[x] == tgt; x++) {
        if (uw[x] < 0) { dels++; dw = -(int64_t)uw[x]; } else { iw += uw[x]; }
      }
      if (dels > 1) { atomicOr(err, 4ull); continue; }       // duplicate deletion
      const int64_t f = row_find(idx, a0, a1, tgt);
      const bool exists = f < a1 && idx[f] == tgt;
      if (dels && (!exists || (int64_t)w[f] != dw)) { atomicOr(err, 2ull); continue; }  // missing edge / weight
      uint8_t kind;
      int64_t nw;
      if (exists) {
        if (dels && iw == 0) { kind = UPD_REMOVED; nw = 0; }
        else { kind = UPD_REWEIGHT; nw = dels ? iw : (int64_t)w[f] + iw; }
      } else {
        kind = UPD_NEW; nw = iw;
      }
      if (nw > INT32_MAX) { atomicOr(err, 1024ull); nw = INT32_MAX; }  // weight beyond int32
      ut[q] = tgt; uw[q] = (int32_t)nw; uk[q] = kind; Rp[q] = R; Np[q] = N;
      R += kind == UPD_REMOVED;
      N += kind == UPD_NEW;
      q++;
    }
    nrec[u] = q - b;
    newdeg[u] = (a1 - a0) - R + N;
  }
}
// Row starts as a bitmap over the entries (for the sortedness check of the
// rows copied as runs).
__global__ void ba_rowstart_k(int64_t n, const int64_t *off, uint32_t *bits) {
  DSTRIDE(u, n) {
    const int64_t a = off[u];
    if (off[u + 1] > a) atomicOr(&bits[a >> 5], 1u << (a & 31));
  }
}
// The entries of untouched rows, copied in runs: every run of untouched rows
// between two touched ones moves by one shift (the length change of the
// touched rows before it).  Each warp takes a tile of 32 x BA_TILE entries;
// lane 0 finds the tile's first run by binary search over the touched rows'
// starts, and each lane walks forward from there.  Also checks that every
// copied row is strictly increasing.
static constexpr int BA_TILE = 16;
__global__ void ba_copy_k(int64_t nnz, int64_t T, const int32_t *trow, const int64_t *off, const int64_t *off2,
                          const int32_t *idx, const int32_t *w, const uint32_t *bits, int64_t nnz2,
                          int32_t *idx2, int32_t *w2, u64 *err) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr int64_t TILE = 32 * BA_TILE;
  for (int64_t t0 = wid * TILE; t0 < nnz; t0 += nwarps * TILE) {
    int64_t k0 = 0;  // touched rows that start at or before t0
    if (lane == 0) {
      int64_t lo = 0, hi = T;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[trow[mid]] <= t0) lo = mid + 1; else hi = mid;
      }
      k0 = lo;
    }
    int64_t k = shfl_i64(k0, 0);
    for (int m = 0; m < BA_TILE; m++) {
      const int64_t e = t0 + (int64_t)m * 32 + lane;
      if (e >= nnz) break;
      while (k < T && off[trow[k]] <= e) k++;
      // e lies in touched row trow[k - 1] if it is before that row's end
      if (k > 0 && e < off[trow[k - 1] + 1]) continue;
      const int64_t r1 = k > 0 ? (int64_t)trow[k - 1] + 1 : 0;   // first row of this run
      const int64_t pos = e + (off2[r1] - off[r1]);
      const int32_t x = idx[e];
      if (e > 0 && !((bits[e >> 5] >> (e & 31)) & 1u) && idx[e - 1] >= x) atomicOr(err, 8ull);
      if (pos < 0 || pos >= nnz2) { atomicOr(err, 8ull); continue; }
      idx2[pos] = x;
      w2[pos] = w[e];
    }
  }
}
// BA_MERGE_LANES lanes per touched row (most touched rows are short, so a
// whole warp per row would leave most lanes idle): every surviving old entry
// goes to its rank among the new row (its position less the removed entries
// before it plus the new ones before it), every new entry likewise.
static constexpr int BA_MERGE_LANES = 8;
__global__ void ba_merge_k(int64_t T, const int32_t *trow, const int64_t *uoff, const int64_t *nrec,
                           const int32_t *ut, const int32_t *uw, const uint8_t *uk, const int32_t *Rp,
                           const int32_t *Np, const int64_t *off, const int32_t *idx, const int32_t *w,
                           const int64_t *off2, int32_t *idx2, int32_t *w2, u64 *err) {
  constexpr int G = BA_MERGE_LANES;
  const int lane = threadIdx.x % G;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t t = wid; t < T; t += nwarps) {
    const int32_t u = trow[t];
    const int64_t a0 = off[u], a1 = off[u + 1];
    const int64_t p0 = uoff[u], nr = nrec[u];
    const int64_t o0 = off2[u], len = off2[u + 1] - o0;
    for (int64_t a = a0 + lane; a < a1; a += G) {
      const int32_t x = idx[a];
      if (a > a0 && idx[a - 1] >= x) { atomicOr(err, 8ull); continue; }
      int64_t lo = 0, hi = nr;                                 // first record with target >= x
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ut[p0 + mid] < x) lo = mid + 1; else hi = mid;
      }
      int64_t rb, nb;
      if (lo < nr) { rb = Rp[p0 + lo]; nb = Np[p0 + lo]; }
      else if (nr > 0) {                                       // after every record
        const int64_t l = p0 + nr - 1;
        rb = Rp[l] + (uk[l] == UPD_REMOVED);
        nb = Np[l] + (uk[l] == UPD_NEW);
      } else { rb = 0; nb = 0; }
      int32_t wt = w[a];
      if (lo < nr && ut[p0 + lo] == x) {
        if (uk[p0 + lo] == UPD_REMOVED) continue;
        wt = uw[p0 + lo];
      }
      const int64_t pos = (a - a0) - rb + nb;
      if (pos < 0 || pos >= len) { atomicOr(err, 8ull); continue; }
      idx2[o0 + pos] = x;
      w2[o0 + pos] = wt;
    }
    for (int64_t q = lane; q < nr; q += G) {
      if (uk[p0 + q] != UPD_NEW) continue;
      const int32_t y = ut[p0 + q];
      const int64_t pos = (row_find(idx, a0, a1, y) - a0) - Rp[p0 + q] + Np[p0 + q];
      if (pos < 0 || pos >= len) { atomicOr(err, 8ull); continue; }
      idx2[o0 + pos] = y;
      w2[o0 + pos] = uw[p0 + q];
    }
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
  // per-row update lists
  cudaMemsetAsync(wk.cnt, 0, (size_t)(n + 1) * sizeof(int64_t), s);
  cudaMemsetAsync(wk.cur, 0, (size_t)(n + 1) * sizeof(int64_t), s);
  if (nd > 0) LK_COUNTED ba_cnt_k<<<gridd(nd, 256), 256, 0, s>>>(nd, ds, dd, wk.cnt);
  if (ni > 0) LK_COUNTED ba_cnt_k<<<gridd(ni, 256), 256, 0, s>>>(ni, is, id, wk.cnt);
  exclusive_scan<int64_t>(wk.cnt, wk.uoff, n, wk.scan_tmp, s);
  if (nd > 0) LK_COUNTED ba_place_k<<<gridd(nd, 256), 256, 0, s>>>(nd, ds, dd, dw, -1, wk.uoff, wk.cur, wk.ut, wk.uw);
  if (ni > 0) LK_COUNTED ba_place_k<<<gridd(ni, 256), 256, 0, s>>>(ni, is, id, iw, 1, wk.uoff, wk.cur, wk.ut, wk.uw);
  // the touched rows, in increasing order
  if (n > 0) LK_COUNTED ba_touched_flag_k<<<gridd(n, 256), 256, 0, s>>>(n, wk.cnt, wk.tflag);
  exclusive_scan<uint8_t>(wk.tflag, wk.tpos, n, wk.scan_tmp, s);
  if (n > 0) LK_COUNTED ba_touched_list_k<<<gridd(n, 256), 256, 0, s>>>(n, wk.tflag, wk.tpos, wk.trow);
  int64_t T = 0;
  cudaMemcpyAsync(&T, wk.tpos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
  // new row lengths: the old ones, then the touched rows' own
  if (n > 0) LK_COUNTED ba_deg_k<<<gridd(n, 256), 256, 0, s>>>(n, off, wk.newdeg);
  if (T > 0)
    LK_COUNTED ba_row_k<<<gridd(T, 128), 128, 0, s>>>(T, wk.trow, wk.uoff, wk.ut, wk.uw, wk.uk, wk.Rp, wk.Np, wk.cnt,
                                                      off, idx, w, wk.newdeg, wk.err);
  exclusive_scan<int64_t>(wk.newdeg, off_out, n, wk.scan_tmp, s);
  int64_t nnz2 = 0;
  cudaMemcpyAsync(&nnz2, off_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&herr, wk.err, sizeof(u64), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
  if (herr) return LEIDEN_EINVAL;
  if (nnz2 > cap_nnz) return LEIDEN_ENOMEM;
  if (nnz > 0) {
    const int64_t words = (nnz + 31) / 32;
    cudaMemsetAsync(wk.bits, 0, (size_t)words * sizeof(uint32_t), s);
    LK_COUNTED ba_rowstart_k<<<gridd(n, 256), 256, 0, s>>>(n, off, wk.bits);
    const int64_t tiles = (nnz + 32 * BA_TILE - 1) / (32 * BA_TILE);
    LK_COUNTED ba_copy_k<<<gridd(tiles * 32, 256, 152 * 64), 256, 0, s>>>(nnz, T, wk.trow, off, off_out, idx, w,
                                                                         wk.bits, nnz2, idx_out, w_out, wk.err);
  }
  if (T > 0)
    LK_COUNTED ba_merge_k<<<gridd(T * BA_MERGE_LANES, 256, 152 * 32), 256, 0, s>>>(T, wk.trow, wk.uoff, wk.cnt, wk.ut, wk.uw,
                                                                      wk.uk, wk.Rp, wk.Np, off, idx, w, off_out,
                                                                      idx_out, w_out, wk.err);
  cudaMemcpyAsync(&herr, wk.err, sizeof(u64), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
  if (herr) return LEIDEN_EINVAL;
  *nnz_out = nnz2;
  return LEIDEN_OK;
}

}  // namespace lk
