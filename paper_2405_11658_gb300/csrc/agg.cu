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
//    shared table, or, for the largest communities, their entries split by
//    target into shared-memory-sized buckets hashed by many blocks (the load
//    imbalance of selective refinement, Sec. 4.4);
// 4. exclusive scan of cdist gives the compact super-vertex offsets; a copy
//    removes the holes.
// Row order inside the super-vertex graph is whatever the tables produced:
// every later phase only sums and compares, so order does not matter.
#include <limits.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

// 1: the bucket path's count pass leaves each pair at its flat position and
// the scatter streams them (0: the scatter walks the member rows again).
#ifndef LK_AGG_PAIR_CACHE
#define LK_AGG_PAIR_CACHE 1
#endif

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

// Flattened walk over the row segments of a warp's lanes: lane l holds a
// segment of cnt entries starting at CSR position rs, incl is the inclusive
// prefix of cnt over the lanes and total its sum.  The warp visits the
// segments' entries 32 at a time, AGG_UNROLL batches in flight (their idx and
// C' loads issued before the first is used), and calls f(target, weight,
// active) warp-uniformly for each batch.
static constexpr int AGG_UNROLL = 4;
template <typename WT, typename F>
__device__ __forceinline__ void walk_segments(const GraphView<WT> &g, const int32_t *C, int64_t rs, int64_t cnt,
                                              int64_t incl, int64_t total, u64 *err, F f, int64_t fbase = 0) {
  const int lane = threadIdx.x & 31;
  for (int64_t t0 = 0; t0 < total; t0 += 32 * AGG_UNROLL) {  // uniform per warp
    int32_t jj[AGG_UNROLL];
    u64 wv[AGG_UNROLL];
#pragma unroll
    for (int u = 0; u < AGG_UNROLL; u++) {
      const int64_t t = t0 + 32 * u + lane;
      // first lane whose inclusive sum exceeds t
      int k = 0;
#pragma unroll
      for (int b = 16; b; b >>= 1) {
        const int64_t v = shfl_i64(incl, k + b - 1);
        if (v <= t) k += b;
      }
      const int64_t sk = shfl_i64(rs, k), ik = shfl_i64(incl, k), dk = shfl_i64(cnt, k);
      jj[u] = -1;
      wv[u] = 0;
      if (t < total) {
        const int64_t e = sk + (t - (ik - dk));
        if (e >= sk && e < sk + dk) { jj[u] = g.idx[e]; wv[u] = (u64)(int64_t)g.w[e]; }
        else atomicOr(err, 64ull);
      }
    }
    int32_t cc[AGG_UNROLL];
#pragma unroll
    for (int u = 0; u < AGG_UNROLL; u++) {
      const bool ok = (uint32_t)jj[u] < (uint32_t)g.n;
      if (!ok && jj[u] != -1) atomicOr(err, 64ull);
      cc[u] = ok ? C[jj[u]] : LEIDEN_EMPTY_KEY;
    }
#pragma unroll
    for (int u = 0; u < AGG_UNROLL; u++) {
      // the entry's position in the walked range (fbase + t), -1 past its end
      const int64_t t = t0 + 32 * u + lane;
      f(cc[u], wv[u], cc[u] != LEIDEN_EMPTY_KEY, t < total ? fbase + t : (int64_t)-1);
    }
  }
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
    walk_segments(g, C, start, deg, incl, total, err, [&](int32_t c, u64 wv, bool act, int64_t) {
      u64 sum = 0;
      if (warp_combine((unsigned long long)(uint32_t)c, act, wv, &sum, scratch)) tadd(keys, vals, mask, sh, c, sum, err);
    });
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

// Block tier: one block per community, table of 2^log2H shared slots.  The
// community's member rows are walked as one flat range spread over all the
// block's threads (a community of a few long super-vertex rows keeps every
// warp busy): up to blockDim.x members at a time, their row starts and the
// inclusive prefix of their degrees in shared memory, each thread finding
// the member of its entry by a binary search over the prefix, AGG_UNROLL
// entries per thread with their idx and C' loads in flight together.
static constexpr int AGG_BLOCK_MAXT = 512;
template <typename WT>
__global__ void __launch_bounds__(AGG_BLOCK_MAXT) agg_block_k(GraphView<WT> g, const int32_t *C, const int32_t *list,
                                                   int64_t nlist, const int64_t *coff, const int64_t *hoff,
                                                   const int32_t *cv, int32_t *hidx, int64_t *hw,
                                                   int64_t *cdist, int64_t *Kout, int log2H, u64 *err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int H = 1 << log2H;
  // dynamic shared memory: the table (2^log2H values, then keys), then per
  // thread a member row start and degree prefix, then the warps' scratch
  const int nt = blockDim.x;
  u64 *vals = reinterpret_cast<u64 *>(smem);
  int32_t *keys = reinterpret_cast<int32_t *>(vals + H);
  int64_t *m_rs = reinterpret_cast<int64_t *>(keys + H);   // row start of each member of the batch
  int64_t *m_incl = m_rs + nt;                             // inclusive prefix of their degrees
  u64 (*wscratch)[32] = reinterpret_cast<u64 (*)[32]>(m_incl + nt);
  __shared__ unsigned long long s_cnt;
  __shared__ int64_t s_ws;
  __shared__ int64_t w_tot[AGG_BLOCK_MAXT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int64_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int32_t c = list[li];
    const int64_t td = hoff[c + 1] - hoff[c];
    int lh = 1;
    while (lh < log2H && ((int64_t)1 << lh) < 2 * td) lh++;
    const int Hc = 1 << lh;
    for (int s = threadIdx.x; s < Hc; s += nt) { keys[s] = LEIDEN_EMPTY_KEY; vals[s] = 0; }
    if (threadIdx.x == 0) { s_cnt = 0; s_ws = 0; }
    const int64_t mb0 = coff[c], mb1 = coff[c + 1];
    for (int64_t mb = mb0; mb < mb1; mb += nt) {
      const int64_t m = mb + threadIdx.x;
      int64_t rs = 0, deg = 0;
      if (m < mb1) {
        const int32_t v = cv[m];
        rs = g.off[v];
        deg = g.off[v + 1] - rs;
      }
      int64_t x = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = shfl_i64(x, (lane - o) & 31);
        if (lane >= o) x += y;
      }
      if (lane == 31) w_tot[warp] = x;
      __syncthreads();   // also: the table is clear, the previous batch is done
      int64_t pre = 0, total = 0;
      for (int q = 0; q < nwarp; q++) {
        const int64_t tq = w_tot[q];
        if (q < warp) pre += tq;
        total += tq;
      }
      m_rs[threadIdx.x] = rs;
      m_incl[threadIdx.x] = pre + x;
      const int nm = (int)(mb1 - mb < nt ? mb1 - mb : nt);
      __syncthreads();
      for (int64_t t0 = 0; t0 < total; t0 += (int64_t)nt * AGG_UNROLL) {  // uniform over the block
        int32_t jj[AGG_UNROLL];
        u64 wv[AGG_UNROLL];
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          const int64_t t = t0 + (int64_t)u * nt + threadIdx.x;
          jj[u] = -1;
          wv[u] = 0;
          if (t < total) {
            // first member whose inclusive prefix exceeds t
            int lo = 0, hi = nm - 1;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (m_incl[mid] > t) hi = mid; else lo = mid + 1;
            }
            const int64_t before = lo ? m_incl[lo - 1] : 0;
            const int64_t e = m_rs[lo] + (t - before);
            jj[u] = g.idx[e];
            wv[u] = (u64)(int64_t)g.w[e];
          }
        }
        int32_t cc[AGG_UNROLL];
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          const bool ok = (uint32_t)jj[u] < (uint32_t)g.n;
          if (!ok && jj[u] != -1) atomicOr(err, 64ull);
          cc[u] = ok ? C[jj[u]] : LEIDEN_EMPTY_KEY;
        }
#pragma unroll
        for (int u = 0; u < AGG_UNROLL; u++) {
          u64 sum = 0;
          if (warp_combine((unsigned long long)(uint32_t)cc[u], cc[u] != LEIDEN_EMPTY_KEY, wv[u], &sum,
                           wscratch[warp]))
            tadd(keys, vals, Hc - 1, 32 - lh, cc[u], sum, err);
        }
      }
      __syncthreads();   // the batch's prefix is read before the next one is written
    }
    if (mb0 == mb1) __syncthreads();
    warp_emit(keys, vals, Hc, 32 * warp, 32 * nwarp, hidx, hw, hoff[c], &s_cnt, &s_ws);
    __syncthreads();
    if (threadIdx.x == 0) { cdist[c] = (int64_t)s_cnt; Kout[c] = s_ws; }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Giant communities (total degree above the block tier).  Their entries are
// partitioned by the hash of the target community into buckets, each sized so
// that its distinct targets fit a shared-memory table, in three passes over
// their member rows (count, scatter) plus one over the buckets (hash, emit):
//   size:    P_k = power of two >= min(tdeg_k, |Gamma|) / BUCKET_KEYS buckets;
//   count:   entries per bucket (warp-combined atomics);
//   scan:    bucket offsets in the scratch arrays (the output graph's idx and
//            w arrays, free until the final compaction writes them);
//   scatter: (target, weight) pairs into their bucket's range of the scratch;
//   hash:    one block per bucket builds its table in shared memory and emits
//            the distinct targets into the community's hole range.
// No hash table lives in DRAM, so no atomic has to go there.
// ---------------------------------------------------------------------------
static constexpr int BUCKET_KEYS = 4096;      // at most this many distinct targets per bucket, on average
static constexpr int64_t AGG_WINDOW = 512;    // flat entries per warp work item
static constexpr uint32_t BUCKET_SLOTS = 6144;  // shared table of a bucket: 3x headroom
static constexpr int BH_UNROLL = 4;              // chunks of 32 pairs in flight per warp

__global__ void agg_bsize_k(const int32_t *list, int64_t nlist, const int64_t *hoff, int64_t nc, int64_t *nbk,
                            int64_t *nwin) {
  GSTRIDE(k, nlist) {
    const int32_t c = list[k];
    const int64_t d = hoff[c + 1] - hoff[c];
    const int64_t cap = d < nc ? d : nc;
    int64_t P = 1;
    while (P * BUCKET_KEYS < cap) P <<= 1;
    nbk[k] = P;
    nwin[k] = (d + AGG_WINDOW - 1) / AGG_WINDOW;
  }
}

// Degree of the member at each position of the community-vertex array, for
// the prefix sums that place every entry of a community in its flat range.
template <typename WT>
__global__ void agg_member_deg_k(GraphView<WT> g, const int32_t *cv, int64_t n, int64_t *mdeg) {
  GSTRIDE(p, n) {
    const int32_t v = cv[p];
    mdeg[p] = g.off[v + 1] - g.off[v];
  }
}

// The warp walks the entries [w0, w1) of one community's flattened rows
// (members cv[p_lo .. p_hi), pdeg = exclusive prefix of their degrees, so the
// community's flat range starts at pdeg[p_lo]) and calls f(target, weight,
// active, flat position) warp-uniformly, 32 entries at a time.
template <typename WT, typename F>
__device__ __forceinline__ void foreach_window(const GraphView<WT> &g, const int32_t *C, const int32_t *cv,
                                               const int64_t *pdeg, int64_t p_lo, int64_t p_hi, int64_t w0,
                                               int64_t w1, u64 *err, F f) {
  const int lane = threadIdx.x & 31;
  // first member whose range reaches past w0
  int64_t lo = p_lo, hi = p_hi - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (pdeg[mid + 1] > w0) hi = mid; else lo = mid + 1;
  }
  for (int64_t pb = lo; pb < p_hi; pb += 32) {
    if (pdeg[pb] >= w1) break;  // same address for every lane: uniform
    const int64_t m = pb + lane;
    int64_t rs = 0, cnt = 0;
    if (m < p_hi) {
      const int64_t fs0 = pdeg[m], fe0 = pdeg[m + 1];
      const int64_t fs = fs0 > w0 ? fs0 : w0, fe = fe0 < w1 ? fe0 : w1;
      if (fe > fs) {
        rs = g.off[cv[m]] + (fs - fs0);
        cnt = fe - fs;
      }
    }
    int64_t incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = shfl_i64(incl, (lane - o) & 31);
      if (lane >= o) incl += y;
    }
    const int64_t total = shfl_i64(incl, 31);
    // the batch's clipped segments are consecutive in the flat range
    const int64_t fb = pdeg[pb] > w0 ? pdeg[pb] : w0;
    walk_segments(g, C, rs, cnt, incl, total, err, f, fb);
  }
}

// Work item b belongs to the last k with offs[k] <= b.
__device__ __forceinline__ int64_t find_k(const int64_t *offs, int64_t n, int64_t b) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t bucket_of(int32_t c, int64_t P) {
  int lp = 0;
  while (((int64_t)1 << lp) < P) lp++;
  return lp ? (int64_t)(hash32(c) >> (32 - lp)) : 0;
}

// PASS = 0: count entries per bucket.  PASS = 1: scatter them.  Work item =
// one warp-sized window of AGG_WINDOW entries of one giant community.  The
// community's own entries (its internal weight, usually most of a giant
// community's rows) are not bucketed: PASS 0 sums them into selfw[k] and the
// hashing block of the bucket that key c falls in adds them as one pair, so
// no bucket holds the bulk of a community.
template <int PASS, typename WT>
__global__ void __launch_bounds__(256) agg_bpass_k(GraphView<WT> g, const int32_t *C, const int32_t *list,
                                                   int64_t nlist, const int64_t *wnoff, const int64_t *nbk,
                                                   const int64_t *bkoff, const int64_t *coff, const int64_t *hoff,
                                                   const int32_t *cv, const int64_t *pdeg, u64 *bcnt,
                                                   const int64_t *bpos, int32_t *skeys, u64 *svals, u64 *selfw,
                                                   u64 *err, int32_t *pk = nullptr, int64_t *pw = nullptr) {
  const int64_t nitems = wnoff[nlist];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ u64 wscr[8][32];  // blocks of 256 threads
  const int64_t w0g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwg = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = w0g; it < nitems; it += nwg) {  // uniform per warp
    const int64_t k = find_k(wnoff, nlist, it);
    const int32_t c = list[k];
    const int64_t fw0 = hoff[c] + (it - wnoff[k]) * AGG_WINDOW;
    const int64_t fw1 = fw0 + AGG_WINDOW < hoff[c + 1] ? fw0 + AGG_WINDOW : hoff[c + 1];
    const int64_t P = nbk[k], base = bkoff[k];
    foreach_window(g, C, cv, pdeg, coff[c], coff[c + 1], fw0, fw1, err, [&](int32_t d, u64 w, bool act0,
                                                                             int64_t fpos) {
      const bool self = act0 && d == c;
      if (PASS == 0) {
        u64 sw = self ? w : 0;
        for (int o = 16; o; o >>= 1) sw += __shfl_xor_sync(FULL_MASK, sw, o);
        if (lane == 0 && sw) atomicAdd(&selfw[k], sw);
      }
      // equal targets within the warp become one pair (hot targets would
      // otherwise fill one bucket); both passes see the same leaders
      u64 wsum = 0;
      const bool act = warp_combine((unsigned long long)(uint32_t)d, act0 && !self, w, &wsum, wscr[warp]);
      w = wsum;
      if (PASS == 0 && pk && fpos >= 0) {
        // the pair at its flat position, for the scatter (none: -1)
        pk[fpos] = act ? d : LEIDEN_EMPTY_KEY;
        pw[fpos] = act ? (int64_t)w : 0;
      }
      const int64_t bk = act ? base + bucket_of(d, P) : -1;
      // lanes of the same bucket share one atomic
      const unsigned am = __ballot_sync(FULL_MASK, act);
      if (act) {
        const unsigned peers = __match_any_sync(am, (unsigned long long)bk);
        const int leader = __ffs(peers) - 1;
        if (PASS == 0) {
          if (lane == leader) atomicAdd(&bcnt[bk], (u64)__popc(peers));
        } else {
          u64 slot0 = 0;
          if (lane == leader) slot0 = atomicAdd(&bcnt[bk], (u64)__popc(peers));
          slot0 = __shfl_sync(peers, slot0, leader);
          const int64_t pos = bpos[bk] + (int64_t)slot0 + __popc(peers & ((1u << lane) - 1u));
          skeys[pos] = d;
          svals[pos] = w;
        }
      }
      __syncwarp();
    });
  }
}

// Scatter of the pairs the count pass left at their flat positions: a
// streamed read of them, instead of a second walk of the member rows with
// their C'[j] gathers.  A warp takes 32 consecutive positions at a time.
__global__ void __launch_bounds__(256) agg_bscatter_k(const int32_t *list, int64_t nlist, const int64_t *wnoff,
                                                      const int64_t *nbk, const int64_t *bkoff,
                                                      const int64_t *hoff, const int32_t *pk, const int64_t *pw,
                                                      u64 *bcnt, const int64_t *bpos, int32_t *skeys,
                                                      u64 *svals) {
  const int64_t nitems = wnoff[nlist];
  const int lane = threadIdx.x & 31;
  const int64_t w0g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwg = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = w0g; it < nitems; it += nwg) {  // uniform per warp
    const int64_t k = find_k(wnoff, nlist, it);
    const int32_t c = list[k];
    const int64_t fw0 = hoff[c] + (it - wnoff[k]) * AGG_WINDOW;
    const int64_t fw1 = fw0 + AGG_WINDOW < hoff[c + 1] ? fw0 + AGG_WINDOW : hoff[c + 1];
    const int64_t P = nbk[k], base = bkoff[k];
    for (int64_t f0 = fw0; f0 < fw1; f0 += 32) {
      const int64_t f = f0 + lane;
      const int32_t d = f < fw1 ? pk[f] : LEIDEN_EMPTY_KEY;
      const bool act = d != LEIDEN_EMPTY_KEY;
      const u64 w = act ? (u64)pw[f] : 0;
      const int64_t bk = act ? base + bucket_of(d, P) : -1;
      const unsigned am = __ballot_sync(FULL_MASK, act);
      if (act) {
        const unsigned peers = __match_any_sync(am, (unsigned long long)bk);
        const int leader = __ffs(peers) - 1;
        u64 slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(&bcnt[bk], (u64)__popc(peers));
        slot0 = __shfl_sync(peers, slot0, leader);
        const int64_t pos = bpos[bk] + (int64_t)slot0 + __popc(peers & ((1u << lane) - 1u));
        skeys[pos] = d;
        svals[pos] = w;
      }
      __syncwarp();
    }
  }
}

// One block per bucket: hash the bucket's pairs in shared memory and emit the
// distinct targets into the community's hole range.  The
// table is cleared once per block; every bucket lists the slots it occupies
// (one shared atomic per warp) and resets exactly those while emitting them,
// so a bucket costs work in proportion to its pairs, not to the table size.
// A bucket reserves its output range with one global atomic, and thread 0
// fetches the next bucket's description while the block emits.
// Owner (index into the giant list) of every bucket, so a hashing block finds
// its bucket's community with one load instead of a binary search.
__global__ void agg_bown_k(const int64_t *bkoff, int64_t nlist, int32_t *bown) {
  GSTRIDE(k, nlist) {
    for (int64_t b = bkoff[k]; b < bkoff[k + 1]; b++) bown[b] = (int32_t)k;
  }
}

struct BucketInfo {
  int64_t p0, p1;
  int32_t c, lp;
  u64 self;   // internal weight, if this bucket is the one key c falls in
};

__device__ __forceinline__ BucketInfo bucket_info(int64_t bk, const int32_t *list, const int32_t *bown,
                                                  const int64_t *nbk, const int64_t *bkoff, const int64_t *bpos,
                                                  const u64 *selfw) {
  BucketInfo b;
  const int32_t k = bown[bk];
  b.p0 = bpos[bk];
  b.p1 = bpos[bk + 1];
  b.c = list[k];
  const int64_t P = nbk[k];
  int lp = 0;
  while (((int64_t)1 << lp) < P) lp++;
  b.lp = lp;
  const u64 sw = selfw[k];
  b.self = (sw && bk - bkoff[k] == bucket_of(b.c, P)) ? sw : 0;
  return b;
}

__global__ void __launch_bounds__(512) agg_bhash_k(const int32_t *list, const int32_t *bown, const int64_t *nbk,
                                                   const int64_t *bkoff, const int64_t *bpos, const int32_t *skeys,
                                                   const u64 *svals, const u64 *selfw, const int64_t *hoff, int32_t *hidx,
                                                   int64_t *hw, int64_t *cdist, int64_t *Kout, int64_t nb,
                                                   u64 *err) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr uint32_t H = BUCKET_SLOTS;
  u64 *vals = reinterpret_cast<u64 *>(smem);
  int32_t *keys = reinterpret_cast<int32_t *>(vals + H);
  uint16_t *used = reinterpret_cast<uint16_t *>(keys + H);
  __shared__ u64 wscratch[16][32];
  __shared__ int64_t s_ws;
  __shared__ unsigned s_nused;
  __shared__ int64_t s_base;
  __shared__ BucketInfo s_b;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (uint32_t x = threadIdx.x; x < H; x += blockDim.x) { keys[x] = LEIDEN_EMPTY_KEY; vals[x] = 0; }
  if (threadIdx.x == 0) {
    s_nused = 0;
    if (blockIdx.x < nb) s_b = bucket_info(blockIdx.x, list, bown, nbk, bkoff, bpos, selfw);
  }
  for (int64_t bk = blockIdx.x; bk < nb; bk += gridDim.x) {
    __syncthreads();
    const BucketInfo b = s_b;
    const int32_t c = b.c;
    const int lp = b.lp;
    // the bucket's keys share their top lp hash bits: index by the next ones
    // (scaled to the table size)
    auto home = [&](int32_t key) -> uint32_t {
      return (uint32_t)(((u64)(uint32_t)(hash32(key) << lp) * H) >> 32);
    };
    // the community's internal weight joins the bucket its own key falls in
    if (threadIdx.x == 0) {
      s_ws = 0;
      if (b.self) {
        const uint32_t sl = home(c);   // the table is empty: the home slot is free
        keys[sl] = c;
        vals[sl] = b.self;
        used[s_nused++] = (uint16_t)sl;
      }
    }
    __syncthreads();
    // BH_UNROLL chunks of 32 pairs per warp iteration: their loads are all in
    // flight before the first is hashed (one chunk at a time leaves the loop
    // waiting on memory latency)
    for (int64_t pb0 = b.p0 + 32 * BH_UNROLL * warp; pb0 < b.p1; pb0 += 32 * BH_UNROLL * (int64_t)nwarp) {
      int32_t dd[BH_UNROLL];
      u64 ww[BH_UNROLL];
#pragma unroll
      for (int u = 0; u < BH_UNROLL; u++) {
        const int64_t pos = pb0 + 32 * u + lane;
        dd[u] = LEIDEN_EMPTY_KEY;
        ww[u] = 0;
        if (pos < b.p1) { dd[u] = skeys[pos]; ww[u] = svals[pos]; }
      }
#pragma unroll
      for (int u = 0; u < BH_UNROLL; u++) {
        const int32_t d = dd[u];
        u64 sum = 0;
        int fresh = -1;
        if (warp_combine((unsigned long long)(uint32_t)d, d != LEIDEN_EMPTY_KEY, ww[u], &sum, wscratch[warp])) {
          uint32_t sl = home(d);
          bool done = false;
          for (uint32_t probe = 0; probe < H && !done; probe++) {
            const int32_t kk = *(volatile int32_t *)&keys[sl];
            if (kk == d) { atomicAdd(&vals[sl], sum); done = true; }
            else if (kk == LEIDEN_EMPTY_KEY) {
              const int32_t old = atomicCAS(&keys[sl], LEIDEN_EMPTY_KEY, d);
              if (old == LEIDEN_EMPTY_KEY || old == d) {
                atomicAdd(&vals[sl], sum);
                if (old == LEIDEN_EMPTY_KEY) fresh = (int)sl;
                done = true;
              }
            }
            sl = sl + 1 == H ? 0 : sl + 1;
          }
          if (!done) atomicOr(err, 16ull);
        }
        // one shared atomic per warp for the slots it occupied
        const unsigned m = __ballot_sync(FULL_MASK, fresh >= 0);
        if (m) {
          const int leader = __ffs(m) - 1;
          unsigned base = 0;
          if (lane == leader) base = atomicAdd(&s_nused, (unsigned)__popc(m));
          base = __shfl_sync(FULL_MASK, base, leader);
          if (fresh >= 0) used[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)fresh;
        }
      }
    }
    __syncthreads();
    const unsigned nused = s_nused;
    // the block's output range: one global atomic per bucket
    if (threadIdx.x == 0) s_base = (int64_t)atomicAdd((u64 *)&cdist[c], (u64)nused);
    // fetch the next bucket's description while the block emits
    const int64_t nbk_next = bk + gridDim.x;
    BucketInfo nx{};
    if (threadIdx.x == 32 && nbk_next < nb) nx = bucket_info(nbk_next, list, bown, nbk, bkoff, bpos, selfw);
    __syncthreads();
    const int64_t out0 = hoff[c] + s_base;
    int64_t ws = 0;
    for (unsigned u = threadIdx.x; u < nused; u += blockDim.x) {
      const uint32_t sl = used[u];
      const int32_t key = keys[sl];
      const int64_t v = (int64_t)vals[sl];
      keys[sl] = LEIDEN_EMPTY_KEY;   // reset on read: clean for the next bucket
      vals[sl] = 0;
      hidx[out0 + u] = key;
      hw[out0 + u] = v;
      ws += v;
    }
    for (int o = 16; o; o >>= 1) ws += shfl_xor_i64(ws, o);
    if (lane == 0 && ws) atomicAdd((u64 *)&s_ws, (u64)ws);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_ws) atomicAdd((u64 *)&Kout[c], (u64)s_ws);
      s_nused = 0;
    }
    if (threadIdx.x == 32) s_b = nx;
  }
}

// ---------------------------------------------------------------------------
// Compaction of the hole ranges into the final CSR.
// ---------------------------------------------------------------------------
// Small communities: each warp takes 32 of them and copies their ranges as
// one flattened range (prefix sums across the lanes, binary search per entry).
__global__ void agg_compact_small_k(const int32_t *list, int64_t nlist, const int64_t *hoff, const int64_t *off2,
                                    const int32_t *hidx, const int64_t *hw, int32_t *idx2, int64_t *w2) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cb = w0 * 32; cb < nlist; cb += nw * 32) {
    const int64_t li = cb + lane;
    int64_t src = 0, dst = 0, len = 0;
    if (li < nlist) {
      const int32_t c = list[li];
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

// Mid-size communities: one block each.
__global__ void agg_compact_block_k(const int32_t *list, int64_t nlist, const int64_t *hoff, const int64_t *off2,
                                    const int32_t *hidx, const int64_t *hw, int32_t *idx2, int64_t *w2) {
  for (int64_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int32_t c = list[li];
    const int64_t src = hoff[c], dst = off2[c], len = off2[c + 1] - dst;
    for (int64_t x = threadIdx.x; x < len; x += blockDim.x) {
      idx2[dst + x] = hidx[src + x];
      w2[dst + x] = hw[src + x];
    }
  }
}

// Giant communities: output lengths in windows of AGG_WINDOW entries, one
// warp per window.
__global__ void agg_cwin_k(const int32_t *list, int64_t nlist, const int64_t *off2, int64_t *nwin) {
  GSTRIDE(k, nlist) {
    const int32_t c = list[k];
    nwin[k] = (off2[c + 1] - off2[c] + AGG_WINDOW - 1) / AGG_WINDOW;
  }
}
__global__ void agg_compact_win_k(const int32_t *list, int64_t nlist, const int64_t *wnoff, const int64_t *hoff,
                                  const int64_t *off2, const int32_t *hidx, const int64_t *hw, int32_t *idx2,
                                  int64_t *w2) {
  const int lane = threadIdx.x & 31;
  const int64_t w0g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwg = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nitems = wnoff[nlist];
  for (int64_t it = w0g; it < nitems; it += nwg) {
    const int64_t k = find_k(wnoff, nlist, it);
    const int32_t c = list[k];
    const int64_t len = off2[c + 1] - off2[c];
    const int64_t x0 = (it - wnoff[k]) * AGG_WINDOW;
    const int64_t x1 = x0 + AGG_WINDOW < len ? x0 + AGG_WINDOW : len;
    const int64_t src = hoff[c], dst = off2[c];
    for (int64_t x = x0 + lane; x < x1; x += 32) {
      idx2[dst + x] = hidx[src + x];
      w2[dst + x] = hw[src + x];
    }
  }
}

// Communities by total degree: a warp with a small or a larger shared table,
// a block, or the bucketed multi-block path for giant ones -- the GPU form of
// the paper's Optimized Aggregation (Sec. 4.4), which keeps one large
// unrefined community from holding up a worker.  uniform = 1 sends every
// community through the multi-block path instead (one method for all sizes,
// for the ablation of that design).
static TierTable agg_tiers(int uniform) {
  TierTable tt{};
  int k = 0;
  tt.t[k++] = {TIER_SKIP, 0, 0, 0, 0};
  if (!uniform) {
    tt.t[k++] = {TIER_GROUP, 48, 32, 7, 256};     // warp, 128 slots
    tt.t[k++] = {TIER_GROUP, 384, 32, 10, 128};   // warp, 1024 slots
    tt.t[k++] = {TIER_BLOCK, 2048, 0, 12, 256};   // block, 4096 slots (48 KB: 4 blocks per SM)
  }
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
  if (n > 0) LK_COUNTED agg_count_k<<<gridn(n, 256), 256, 0, s>>>(n, g.off, C, wk.ccount, wk.ctdeg);
  exclusive_scan<int64_t>(wk.ccount, wk.coff, nc, wk.scan_tmp, s);
  exclusive_scan<int64_t>(wk.ctdeg, wk.hoff, nc, wk.scan_tmp, s);
  if (n > 0) LK_COUNTED agg_place_k<<<gridn(n, 256), 256, 0, s>>>(n, C, wk.coff, wk.ccur, wk.cv);

  const TierTable tt = agg_tiers(wk.uniform);
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
        LK_COUNTED agg_warp_k<7, WT><<<blocks, T.threads, smem, s>>>(g, C, list, nl, wk.coff, wk.hoff, wk.cv, wk.hidx,
                                                          wk.hw, wk.cdist, Kout, err);
      } else {
        auto k = agg_warp_k<10, WT>;
        ensure_smem((const void *)k, smem);
        LK_COUNTED k<<<blocks, T.threads, smem, s>>>(g, C, list, nl, wk.coff, wk.hoff, wk.cv, wk.hidx, wk.hw,
                                          wk.cdist, Kout, err);
      }
    } else if (T.kind == TIER_BLOCK) {
      // table, member batch (16 bytes a thread), combine scratch (256 bytes a warp)
      const size_t smem = (size_t)(1u << T.log2H) * 12 + (size_t)T.threads * 16 + (size_t)(T.threads / 32) * 256;
      auto k = agg_block_k<WT>;
      ensure_smem((const void *)k, smem);
      const int64_t cap = resident_blocks((const void *)k, T.threads, smem, wk.sms);
      int64_t blocks = nl < cap ? nl : cap;
      LK_COUNTED k<<<(unsigned)blocks, T.threads, smem, s>>>(g, C, list, nl, wk.coff, wk.hoff, wk.cv, wk.hidx, wk.hw,
                                                  wk.cdist, Kout, T.log2H, err);
    } else {
      // giant communities: buckets sized for a shared-memory table
      int64_t *nbk = wk.off2tmp;                    // [nl]   buckets per community
      int64_t *bkoff = wk.off2tmp + (nl + 1);       // [nl+1] bucket index offsets
      int64_t *nwin = wk.off2tmp + 2 * (nl + 1);    // [nl]   entry windows
      int64_t *wnoff = wk.off2tmp + 3 * (nl + 1);   // [nl+1]
      LK_COUNTED agg_bsize_k<<<gridn(nl, 256), 256, 0, s>>>(list, nl, wk.hoff, nc, nbk, nwin);
      exclusive_scan<int64_t>(nbk, bkoff, nl, wk.scan_tmp, s);
      exclusive_scan<int64_t>(nwin, wnoff, nl, wk.scan_tmp, s);
      // member-degree prefix over the community-vertex array: pdeg[coff[c]] =
      // hoff[c], so every community's entries form one flat range
      int64_t *mdeg = wk.ccur;      // free after the placement
      int64_t *pdeg = wk.scanned;   // free after the tier lists were read
      LK_COUNTED agg_member_deg_k<WT><<<gridn(n, 256), 256, 0, s>>>(g, wk.cv, n, mdeg);
      exclusive_scan<int64_t>(mdeg, pdeg, n, wk.scan_tmp, s);
      cudaMemcpyAsync(&wk.h_koff[MAX_TIERS + 1], bkoff + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return LEIDEN_ECUDA;
      const int64_t nb = wk.h_koff[MAX_TIERS + 1];
      if (nb + 1 > wk.bcap) return LEIDEN_ENOMEM;
      cudaMemsetAsync(wk.bcnt, 0, (size_t)(nb + 1) * sizeof(u64), s);
      const unsigned grid = (unsigned)(wk.sms * 16);
      u64 *selfw = reinterpret_cast<u64 *>(wk.off2tmp + 4 * (nl + 1));   // [nl] internal weight
      cudaMemsetAsync(selfw, 0, (size_t)nl * sizeof(u64), s);
      // the count pass leaves each entry's pair (after the warp combine) at its
      // flat position in the communities' hole ranges of hidx / hw, which
      // the bucket hash only writes afterwards
      int32_t *pk = LK_AGG_PAIR_CACHE ? wk.hidx : nullptr;
      int64_t *pw = LK_AGG_PAIR_CACHE ? wk.hw : nullptr;
      LK_COUNTED agg_bpass_k<0, WT><<<grid, 256, 0, s>>>(g, C, list, nl, wnoff, nbk, bkoff, wk.coff, wk.hoff, wk.cv, pdeg,
                                               wk.bcnt, nullptr, nullptr, nullptr, selfw, err, pk, pw);
      exclusive_scan<int64_t>(reinterpret_cast<const int64_t *>(wk.bcnt), wk.bpos, nb, wk.scan_tmp, s);
      cudaMemsetAsync(wk.bcnt, 0, (size_t)(nb + 1) * sizeof(u64), s);
      // the bucket ranges tile [0, sum of the listed total degrees) of the
      // output graph's idx / w arrays, which the compaction below only writes
      // after the buckets are hashed (the scratch needs no clearing then)
      u64 *svals = reinterpret_cast<u64 *>(w2);
      if (LK_AGG_PAIR_CACHE)
        LK_COUNTED agg_bscatter_k<<<grid, 256, 0, s>>>(list, nl, wnoff, nbk, bkoff, wk.hoff, pk, pw, wk.bcnt, wk.bpos,
                                                       idx2, svals);
      else
        LK_COUNTED agg_bpass_k<1, WT><<<grid, 256, 0, s>>>(g, C, list, nl, wnoff, nbk, bkoff, wk.coff, wk.hoff, wk.cv,
                                                 pdeg, wk.bcnt, wk.bpos, idx2, svals, selfw, err);
      const size_t smem = (size_t)BUCKET_SLOTS * (12 + 2);
      ensure_smem((const void *)agg_bhash_k, smem);
      // the bucket counters are free after the scatter: they hold the owners
      int32_t *bown = reinterpret_cast<int32_t *>(wk.bcnt);
      LK_COUNTED agg_bown_k<<<gridn(nl, 256), 256, 0, s>>>(bkoff, nl, bown);
      LK_COUNTED agg_bhash_k<<<(unsigned)(wk.sms * 2), 512, smem, s>>>(list, bown, nbk, bkoff, wk.bpos, idx2,
                                                            svals, selfw, wk.hoff, wk.hidx, wk.hw, wk.cdist, Kout,
                                                            nb, err);
    }
  }
  exclusive_scan<int64_t>(wk.cdist, off2, nc, wk.scan_tmp, s);
  cudaMemcpyAsync(nnz2, off2 + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  for (int t = 1; t < tt.ntiers; t++) {
    const int32_t *list = wk.clist + koff[t];
    const int64_t nl = koff[t + 1] - koff[t];
    if (nl <= 0) continue;
    if (tt.t[t].kind == TIER_GROUP)
      LK_COUNTED agg_compact_small_k<<<gridn(nl, 256, (int64_t)wk.sms * 32), 256, 0, s>>>(list, nl, wk.hoff, off2, wk.hidx,
                                                                              wk.hw, idx2, w2);
    else if (tt.t[t].kind == TIER_BLOCK)
      LK_COUNTED agg_compact_block_k<<<(unsigned)(nl < wk.sms * 8 ? nl : wk.sms * 8), 256, 0, s>>>(list, nl, wk.hoff, off2,
                                                                                      wk.hidx, wk.hw, idx2, w2);
    else {
      int64_t *nwin = wk.off2tmp;
      int64_t *wnoff = wk.off2tmp + (nl + 1);
      LK_COUNTED agg_cwin_k<<<gridn(nl, 256), 256, 0, s>>>(list, nl, off2, nwin);
      exclusive_scan<int64_t>(nwin, wnoff, nl, wk.scan_tmp, s);
      LK_COUNTED agg_compact_win_k<<<(unsigned)(wk.sms * 16), 256, 0, s>>>(list, nl, wnoff, wk.hoff, off2, wk.hidx, wk.hw,
                                                                 idx2, w2);
    }
  }
  return 0;
}

template int aggregate<int32_t>(GraphView<int32_t>, const int32_t *, int64_t, int64_t *, int32_t *,
                                int64_t *, int64_t *, const AggWork &, cudaStream_t);
template int aggregate<int64_t>(GraphView<int64_t>, const int32_t *, int64_t, int64_t *, int32_t *,
                                int64_t *, int64_t *, const AggWork &, cudaStream_t);

}  // namespace lk
