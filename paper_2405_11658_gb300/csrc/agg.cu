// agg.cu -- aggregation phase (Alg. leidenag) on sm_103a.
//
// 1. countCommunityVertices and communityTotalDegree by atomics, two
//    exclusive scans (community-vertex offsets coff, super-vertex offsets
//    hoff "with holes", sized by total degree);
// 2. community-vertex CSR cv by atomic placement;
// 3. per community, scanCommunities with self = true over every member row
//    into a hashtable of (neighbour community d, summed weight); the entries
//    land in the community's hole range and cdist[c] counts them.  Work is
//    bucketed by total degree: a warp with a shared table, a block with a
//    shared table, or many blocks sharing a table in global scratch for the
//    largest communities (the load imbalance of selective refinement,
//    Sec. 4.4);
// 4. exclusive scan of cdist gives the compact super-vertex offsets; a copy
//    removes the holes.
// Row order inside the super-vertex graph is whatever the tables produced:
// every later phase only sums and compares, so order does not matter.
#include <limits.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lk {

static inline unsigned gridn(int64_t n, int threads, int64_t cap = 1 << 20) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}
#define GSTRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void agg_count_k(int64_t n, const int64_t *off, const int32_t *C, int64_t *cnt, int64_t *tdeg) {
  GSTRIDE(i, n) {
    const int32_t c = C[i];
    atomicAdd((u64 *)&cnt[c], 1ull);
    const int64_t d = off[i + 1] - off[i];
    if (d) atomicAdd((u64 *)&tdeg[c], (u64)d);
  }
}
__global__ void agg_place_k(int64_t n, const int32_t *C, const int64_t *coff, int64_t *cur, int32_t *cv) {
  GSTRIDE(i, n) {
    const int32_t c = C[i];
    const int64_t pos = coff[c] + (int64_t)atomicAdd((u64 *)&cur[c], 1ull);
    cv[pos] = (int32_t)i;
  }
}

// Probing is bounded by the table size: a full table (impossible when the
// table has at least twice as many slots as inserted entries) sets *err and
// drops the entry instead of spinning.
__device__ __forceinline__ void tadd(int32_t *keys, u64 *vals, uint32_t mask, int sh, int32_t c, u64 w,
                                     u64 *err) {
  uint32_t s = hash32(c) >> sh;
  for (uint32_t probe = 0; probe <= mask; probe++) {
    int32_t k = *(volatile int32_t *)&keys[s];
    if (k == c) { atomicAdd(&vals[s], w); return; }
    if (k == LEIDEN_EMPTY_KEY) {
      int32_t old = atomicCAS(&keys[s], LEIDEN_EMPTY_KEY, c);
      if (old == LEIDEN_EMPTY_KEY || old == c) { atomicAdd(&vals[s], w); return; }
    }
    s = (s + 1) & mask;
  }
  atomicOr(err, 16ull);
}

// The warp walks the rows of members cv[m0 .. m1) as one flattened range:
// each batch of 32 members is prefix-summed across the lanes, and every lane
// finds the member of its entry by a binary search over the shuffled sums.
// Every loop that contains a shuffle is uniform across the warp.
template <typename WT>
__device__ __forceinline__ void warp_rows_into_table(const GraphView<WT> &g, const int32_t *C,
                                                     const int32_t *cv, int64_t m0, int64_t m1,
                                                     int64_t mstep, int32_t *keys, u64 *vals,
                                                     uint32_t mask, int sh, u64 *err, u64 *scratch) {
  const int lane = threadIdx.x & 31;
  for (int64_t mb = m0; mb < m1; mb += mstep) {
    const int64_t m = mb + lane;
    int64_t start = 0, deg = 0;
    if (m < m1) {
      const int32_t v = cv[m];
      start = g.off[v];
      deg = g.off[v + 1] - start;
    }
    int64_t incl = deg;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = shfl_i64(incl, (lane - o) & 31);
      if (lane >= o) incl += y;
    }
    const int64_t total = shfl_i64(incl, 31);
    for (int64_t t0 = 0; t0 < total; t0 += 32) {
      const int64_t t = t0 + lane;
      // first lane whose inclusive sum exceeds t
      int k = 0;
#pragma unroll
      for (int b = 16; b; b >>= 1) {
        const int64_t v = shfl_i64(incl, k + b - 1);
        if (v <= t) k += b;
      }
      const int64_t sk = shfl_i64(start, k);
      const int64_t ik = shfl_i64(incl, k);
      const int64_t dk = shfl_i64(deg, k);
      int32_t c = LEIDEN_EMPTY_KEY;
      u64 wv = 0;
      if (t < total) {
        const int64_t e = sk + (t - (ik - dk));
        const int32_t j = (e >= sk && e < sk + dk) ? g.idx[e] : -1;
        if ((uint32_t)j < (uint32_t)g.n) { c = C[j]; wv = (u64)(int64_t)g.w[e]; }
        else atomicOr(err, 64ull);
      }
      u64 sum = 0;
      if (warp_combine((unsigned long long)(uint32_t)c, c != LEIDEN_EMPTY_KEY, wv, &sum, scratch))
        tadd(keys, vals, mask, sh, c, sum, err);
    }
  }
}

// Emit the occupied slots of a table into [base, ...), warp-cooperative;
// returns (count, weight sum) in lane 0 of each participating warp via the
// shared counters.
__device__ __forceinline__ void warp_emit(const int32_t *keys, const u64 *vals, int64_t H,
                                          int64_t sbeg, int64_t sstep, int32_t *hidx, int64_t *hw,
                                          int64_t base, unsigned long long *cnt, int64_t *wsum) {
  const int lane = threadIdx.x & 31;
  int64_t ws = 0;
  for (int64_t s0 = sbeg; s0 < H; s0 += sstep) {
    const int64_t s = s0 + lane;
    const int32_t k = s < H ? keys[s] : LEIDEN_EMPTY_KEY;
    const bool occ = k != LEIDEN_EMPTY_KEY;
    const u64 pos = warp_reserve(cnt, occ);
    if (occ) {
      const int64_t v = (int64_t)vals[s];
      hidx[base + (int64_t)pos] = k;
      hw[base + (int64_t)pos] = v;
      ws += v;
    }
  }
  for (int o = 16; o; o >>= 1) ws += shfl_xor_i64(ws, o);
  if (lane == 0 && ws) atomicAdd((u64 *)wsum, (u64)ws);
}

// Warp tier: one warp per community, table of 2^LOG2H shared slots.
template <int LOG2H, typename WT>
__global__ void __launch_bounds__(256) agg_warp_k(GraphView<WT> g, const int32_t *C, const int32_t *list,
                                                  int64_t nlist, const int64_t *coff, const int64_t *hoff,
                                                  const int32_t *cv, int32_t *hidx, int64_t *hw,
                                                  int64_t *cdist, int64_t *Kout, u64 *err) {
  constexpr int H = 1 << LOG2H;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  u64 *vals = reinterpret_cast<u64 *>(smem) + (size_t)warp * H;
  int32_t *keys = reinterpret_cast<int32_t *>(reinterpret_cast<u64 *>(smem) + (size_t)wpb * H) + (size_t)warp * H;
  __shared__ unsigned long long s_cnt[8];
  __shared__ int64_t s_ws[8];
  __shared__ u64 wscratch[8][32];
  const int64_t w0 = (int64_t)blockIdx.x * wpb + warp, nw = (int64_t)gridDim.x * wpb;
  for (int64_t li = w0; li < nlist; li += nw) {
    const int32_t c = list[li];
    // table sized for this community: 2^lh >= 2 * total degree, lh <= LOG2H
    const int64_t td = hoff[c + 1] - hoff[c];
    int lh = 1;
    while (lh < LOG2H && ((int64_t)1 << lh) < 2 * td) lh++;
    const int Hc = 1 << lh;
    for (int s = lane; s < Hc; s += 32) { keys[s] = LEIDEN_EMPTY_KEY; vals[s] = 0; }
    if (lane == 0) { s_cnt[warp] = 0; s_ws[warp] = 0; }
    __syncwarp();
    warp_rows_into_table(g, C, cv, coff[c], coff[c + 1], 32, keys, vals, Hc - 1, 32 - lh, err, wscratch[warp]);
    __syncwarp();
    warp_emit(keys, vals, Hc, 0, 32, hidx, hw, hoff[c], &s_cnt[warp], &s_ws[warp]);
    __syncwarp();
    if (lane == 0) { cdist[c] = (int64_t)s_cnt[warp]; Kout[c] = s_ws[warp]; }
    __syncwarp();
  }
}

// Block tier: one block per community, table of 2^log2H shared slots.
template <typename WT>
__global__ void __launch_bounds__(512) agg_block_k(GraphView<WT> g, const int32_t *C, const int32_t *list,
                                                   int64_t nlist, const int64_t *coff, const int64_t *hoff,
                                                   const int32_t *cv, int32_t *hidx, int64_t *hw,
                                                   int64_t *cdist, int64_t *Kout, int log2H, u64 *err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int H = 1 << log2H;
  u64 *vals = reinterpret_cast<u64 *>(smem);
  int32_t *keys = reinterpret_cast<int32_t *>(vals + H);
  __shared__ unsigned long long s_cnt;
  __shared__ int64_t s_ws;
  __shared__ u64 wscratch[16][32];
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int64_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int32_t c = list[li];
    const int64_t td = hoff[c + 1] - hoff[c];
    int lh = 1;
    while (lh < log2H && ((int64_t)1 << lh) < 2 * td) lh++;
    const int Hc = 1 << lh;
    for (int s = threadIdx.x; s < Hc; s += blockDim.x) { keys[s] = LEIDEN_EMPTY_KEY; vals[s] = 0; }
    if (threadIdx.x == 0) { s_cnt = 0; s_ws = 0; }
    __syncthreads();
    warp_rows_into_table(g, C, cv, coff[c] + 32 * warp, coff[c + 1], 32 * nwarp, keys, vals, Hc - 1,
                         32 - lh, err, wscratch[warp]);
    __syncthreads();
    warp_emit(keys, vals, Hc, 32 * warp, 32 * nwarp, hidx, hw, hoff[c], &s_cnt, &s_ws);
    __syncthreads();
    if (threadIdx.x == 0) { cdist[c] = (int64_t)s_cnt; Kout[c] = s_ws; }
    __syncthreads();
  }
}

// Global tier, step 1: per listed community, table slots (a power of two >=
// 2 * min(total degree, |Gamma|) and >= 4096: the community has at most that
// many distinct neighbour communities), member batches of 256, and 4096-slot
// drain chunks.
__global__ void agg_gsize_k(const int32_t *list, int64_t nlist, const int64_t *hoff, const int64_t *coff,
                            int64_t nc, int64_t *tsz, int64_t *nb, int64_t *nch) {
  GSTRIDE(k, nlist) {
    const int32_t c = list[k];
    const int64_t d = hoff[c + 1] - hoff[c];
    const int64_t cap = d < nc ? d : nc;
    int64_t h = HUB_TABLE_MIN;
    while (h < 2 * cap) h <<= 1;
    tsz[k] = h;
    nb[k] = (coff[c + 1] - coff[c] + 255) / 256;
    nch[k] = h / HUB_TABLE_MIN;
  }
}

// Global tier, step 2: every block takes one batch of 256 members of one
// community (found by binary search over the batch offsets) and adds their
// rows to the community's table in global scratch.
template <typename WT>
__global__ void __launch_bounds__(256) agg_ginsert_k(GraphView<WT> g, const int32_t *C, const int32_t *list,
                                                     int64_t k0, int64_t k1, const int64_t *boff,
                                                     const int64_t *tbase, const int64_t *tsz,
                                                     const int64_t *coff, const int32_t *cv,
                                                     int32_t *gkeys, u64 *gvals, u64 *err) {
  __shared__ u64 wscratch[8][32];
  const int64_t nitems = boff[k1] - boff[k0];
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int64_t b = boff[k0] + item;
    int64_t lo = k0, hi = k1 - 1;  // last k with boff[k] <= b
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (boff[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const int64_t k = lo;
    const int32_t c = list[k];
    const int64_t mfirst = coff[c] + (b - boff[k]) * 256;
    int64_t mlast = mfirst + 256;
    if (mlast > coff[c + 1]) mlast = coff[c + 1];
    const int64_t H = tsz[k];
    int lh = 0;
    while (((int64_t)1 << lh) < H) lh++;
    int32_t *keys = gkeys + (tbase[k] - tbase[k0]);
    u64 *vals = gvals + (tbase[k] - tbase[k0]);
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    warp_rows_into_table(g, C, cv, mfirst + 32 * warp, mlast, 32 * nwarp, keys, vals,
                         (uint32_t)(H - 1), 32 - lh, err, wscratch[warp]);
  }
}

// Global tier, step 3: every block drains one 4096-slot chunk of one table
// into the community's hole range (positions reserved with atomics on the
// community's entry count) and resets the slots it read, leaving the scratch
// empty for its next user.
__global__ void __launch_bounds__(256) agg_gemit_k(const int32_t *list, int64_t k0, int64_t k1,
                                                   const int64_t *choff, const int64_t *tbase,
                                                   const int64_t *hoff, int32_t *gkeys, u64 *gvals,
                                                   int32_t *hidx, int64_t *hw, int64_t *cdist, int64_t *Kout) {
  const int64_t nitems = choff[k1] - choff[k0];
  const int lane = threadIdx.x & 31;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int64_t b = choff[k0] + item;
    int64_t lo = k0, hi = k1 - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (choff[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const int64_t k = lo;
    const int32_t c = list[k];
    const int64_t s0 = (tbase[k] - tbase[k0]) + (b - choff[k]) * HUB_TABLE_MIN;
    int64_t ws = 0;
    for (int64_t x = threadIdx.x; x < HUB_TABLE_MIN; x += blockDim.x) {  // uniform per warp
      const int64_t sl = s0 + x;
      const int32_t key = gkeys[sl];
      const bool occ = key != LEIDEN_EMPTY_KEY;
      const u64 pos = warp_reserve((u64 *)&cdist[c], occ);
      if (occ) {
        const int64_t v = (int64_t)gvals[sl];
        gkeys[sl] = LEIDEN_EMPTY_KEY;
        gvals[sl] = 0;
        hidx[hoff[c] + (int64_t)pos] = key;
        hw[hoff[c] + (int64_t)pos] = v;
        ws += v;
      }
    }
    for (int o = 16; o; o >>= 1) ws += shfl_xor_i64(ws, o);
    if (lane == 0 && ws) atomicAdd((u64 *)&Kout[c], (u64)ws);
  }
}

// Compaction: each warp takes 32 communities and copies their hole ranges
// to the compact CSR as one flattened range (prefix sums across the lanes,
// binary search per entry), so short rows still move in full warps.
__global__ void agg_compact_k(int64_t nc, const int64_t *hoff, const int64_t *off2, const int32_t *hidx,
                              const int64_t *hw, int32_t *idx2, int64_t *w2) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cb = w0 * 32; cb < nc; cb += nw * 32) {
    const int64_t c = cb + lane;
    int64_t src = 0, dst = 0, len = 0;
    if (c < nc) {
      src = hoff[c];
      dst = off2[c];
      len = off2[c + 1] - dst;
    }
    int64_t incl = len;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = shfl_i64(incl, (lane - o) & 31);
      if (lane >= o) incl += y;
    }
    const int64_t total = shfl_i64(incl, 31);
    for (int64_t t0 = 0; t0 < total; t0 += 32) {
      const int64_t t = t0 + lane;
      int k = 0;
#pragma unroll
      for (int b = 16; b; b >>= 1) {
        const int64_t v = shfl_i64(incl, k + b - 1);
        if (v <= t) k += b;
      }
      const int64_t sk = shfl_i64(src, k), dk = shfl_i64(dst, k);
      const int64_t ik = shfl_i64(incl, k), lk = shfl_i64(len, k);
      if (t < total) {
        const int64_t x = t - (ik - lk);
        idx2[dk + x] = hidx[sk + x];
        w2[dk + x] = hw[sk + x];
      }
    }
  }
}

static TierTable agg_tiers() {
  TierTable tt{};
  int k = 0;
  tt.t[k++] = {TIER_SKIP, 0, 0, 0, 0};
  tt.t[k++] = {TIER_GROUP, 48, 32, 7, 256};     // warp, 128 slots
  tt.t[k++] = {TIER_GROUP, 384, 32, 10, 128};   // warp, 1024 slots
  tt.t[k++] = {TIER_BLOCK, 2048, 0, 12, 256};   // block, 4096 slots (48 KB: 4 blocks per SM)
  tt.t[k++] = {TIER_GLOBAL, INT64_MAX, 0, 0, 256};
  tt.ntiers = k;
  return tt;
}

template <typename WT>
int aggregate(GraphView<WT> g, const int32_t *C, int64_t nc, int64_t *off2, int32_t *idx2,
              int64_t *w2, int64_t *nnz2, const AggWork &wk, cudaStream_t s) {
  const int64_t n = g.n;
  cudaMemsetAsync(wk.ccount, 0, (size_t)(nc + 1) * sizeof(int64_t), s);
  cudaMemsetAsync(wk.ctdeg, 0, (size_t)(nc + 1) * sizeof(int64_t), s);
  cudaMemsetAsync(wk.ccur, 0, (size_t)(nc + 1) * sizeof(int64_t), s);
  cudaMemsetAsync(wk.cdist, 0, (size_t)(nc + 1) * sizeof(int64_t), s);
  if (n > 0) agg_count_k<<<gridn(n, 256), 256, 0, s>>>(n, g.off, C, wk.ccount, wk.ctdeg);
  exclusive_scan<int64_t>(wk.ccount, wk.coff, nc, wk.scan_tmp, s);
  exclusive_scan<int64_t>(wk.ctdeg, wk.hoff, nc, wk.scan_tmp, s);
  if (n > 0) agg_place_k<<<gridn(n, 256), 256, 0, s>>>(n, C, wk.coff, wk.ccur, wk.cv);

  const TierTable tt = agg_tiers();
  launch_buckets(wk.hoff, nc, 0, tt, wk.clist, wk.blockhist, wk.scanned, wk.koff_dev, wk.scan_tmp, s);
  cudaMemcpyAsync(wk.h_koff, wk.koff_dev, (size_t)(tt.ntiers + 1) * sizeof(int64_t),
                  cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
  int64_t koff[MAX_TIERS + 1];
  for (int t = 0; t <= tt.ntiers; t++) koff[t] = wk.h_koff[t];

  int64_t *Kout = wk.Kout;
  u64 *err = &wk.ctr[CTR_ERROR];
  cudaMemsetAsync(Kout, 0, (size_t)(nc + 1) * sizeof(int64_t), s);
  for (int t = 1; t < tt.ntiers; t++) {
    const Tier &T = tt.t[t];
    const int32_t *list = wk.clist + koff[t];
    const int64_t nl = koff[t + 1] - koff[t];
    if (nl <= 0) continue;
    if (T.kind == TIER_GROUP) {
      const size_t smem = (size_t)(T.threads / 32) * (1u << T.log2H) * 12;
      const unsigned blocks = gridn(nl * 32, T.threads, (int64_t)wk.sms * 16);
      if (T.log2H == 7) {
        agg_warp_k<7, WT><<<blocks, T.threads, smem, s>>>(g, C, list, nl, wk.coff, wk.hoff, wk.cv, wk.hidx,
                                                          wk.hw, wk.cdist, Kout, err);
      } else {
        auto k = agg_warp_k<10, WT>;
        ensure_smem((const void *)k, smem);
        k<<<blocks, T.threads, smem, s>>>(g, C, list, nl, wk.coff, wk.hoff, wk.cv, wk.hidx, wk.hw,
                                          wk.cdist, Kout, err);
      }
    } else if (T.kind == TIER_BLOCK) {
      const size_t smem = (size_t)(1u << T.log2H) * 12;
      auto k = agg_block_k<WT>;
      ensure_smem((const void *)k, smem);
      int64_t blocks = nl < (int64_t)wk.sms * 4 ? nl : (int64_t)wk.sms * 4;
      k<<<(unsigned)blocks, T.threads, smem, s>>>(g, C, list, nl, wk.coff, wk.hoff, wk.cv, wk.hidx, wk.hw,
                                                  wk.cdist, Kout, T.log2H, err);
    } else {
      // table sizes, member batches and drain chunks of the listed communities
      int64_t *tsz = wk.off2tmp;                    // [nl]
      int64_t *tbase = wk.off2tmp + (nl + 1);       // [nl+1]
      int64_t *nb = wk.off2tmp + 2 * (nl + 1);      // [nl]
      int64_t *boff = wk.off2tmp + 3 * (nl + 1);    // [nl+1]
      int64_t *nch = wk.off2tmp + 4 * (nl + 1);     // [nl]
      int64_t *choff = wk.off2tmp + 5 * (nl + 1);   // [nl+1]
      agg_gsize_k<<<gridn(nl, 256), 256, 0, s>>>(list, nl, wk.hoff, wk.coff, nc, tsz, nb, nch);
      exclusive_scan<int64_t>(tsz, tbase, nl, wk.scan_tmp, s);
      exclusive_scan<int64_t>(nb, boff, nl, wk.scan_tmp, s);
      exclusive_scan<int64_t>(nch, choff, nl, wk.scan_tmp, s);
      // Rounds: the tables of one round fit in a slot budget sized to stay
      // resident in L2, so the insert atomics do not go to DRAM (a single
      // table larger than the budget gets a round of its own).
      cudaMemcpyAsync(&wk.h_koff[MAX_TIERS + 1], tbase + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
      const int64_t total_slots = wk.h_koff[MAX_TIERS + 1];
      const int64_t budget = (LK_AGG_ROUND_SLOTS > 0 && LK_AGG_ROUND_SLOTS < wk.gcap) ? LK_AGG_ROUND_SLOTS : wk.gcap;
      std::vector<int64_t> h_tb;
      if (total_slots > budget) {
        h_tb.resize(nl + 1);
        if (cudaMemcpy(h_tb.data(), tbase, (nl + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
          return LEIDEN_ECUDA;
      }
      int64_t k0 = 0;
      while (k0 < nl) {
        int64_t k1 = nl;
        if (total_slots > budget) {
          k1 = k0 + 1;
          while (k1 < nl && h_tb[k1 + 1] - h_tb[k0] <= budget) k1++;
          if (h_tb[k1] - h_tb[k0] > wk.gcap) return LEIDEN_ENOMEM;
        }
        // scratch tables are empty on entry (every user drains and resets them)
        agg_ginsert_k<WT><<<(unsigned)(wk.sms * 8), 256, 0, s>>>(g, C, list, k0, k1, boff, tbase, tsz, wk.coff,
                                                                 wk.cv, wk.gkeys, wk.gvals, err);
        agg_gemit_k<<<(unsigned)(wk.sms * 8), 256, 0, s>>>(list, k0, k1, choff, tbase, wk.hoff, wk.gkeys, wk.gvals,
                                                            wk.hidx, wk.hw, wk.cdist, Kout);
        k0 = k1;
      }
    }
  }
  exclusive_scan<int64_t>(wk.cdist, off2, nc, wk.scan_tmp, s);
  cudaMemcpyAsync(nnz2, off2 + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  agg_compact_k<<<gridn(nc * 32, 256, (int64_t)wk.sms * 32), 256, 0, s>>>(nc, wk.hoff, off2, wk.hidx, wk.hw,
                                                                        idx2, w2);
  return 0;
}

template int aggregate<int32_t>(GraphView<int32_t>, const int32_t *, int64_t, int64_t *, int32_t *,
                                int64_t *, int64_t *, const AggWork &, cudaStream_t);
template int aggregate<int64_t>(GraphView<int64_t>, const int32_t *, int64_t, int64_t *, int32_t *,
                                int64_t *, int64_t *, const AggWork &, cudaStream_t);

}  // namespace lk
