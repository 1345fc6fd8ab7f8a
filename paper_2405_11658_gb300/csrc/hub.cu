// hub.cu -- local-move (Alg. leidenlm) and refinement (Alg. leidenre)
// decisions for rows too long for one block's shared memory ("hub" rows of
// power-law graphs and of their super-vertex graphs).
//
// One hub row is spread over many blocks so that no single block serialises
// a row of 10^5 - 10^7 entries:
//   prep   (1 block)  eligibility, per-hub table size 2^k >= 2 min(deg, |V'|),
//                     and exclusive scans of table sizes and work counts;
//   insert (grid)     work item = (hub, 4096-entry chunk of its row): add
//                     (C'[j], w) to the hub's table in global scratch;
//   scan   (grid)     work item = (hub, 4096-slot chunk of its table): best
//                     candidate of the chunk and the hub's own-community
//                     weight; every slot read is reset to empty, so the
//                     scratch is clean again for the next user;
//   final  (per hub)  reduce the chunks, Eq. 2 (scaled) and the move rule,
//                     then propose (DET) or commit (ASYNC).
// Work counts stay on the device: grids are fixed and stride over them.
#include <limits.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace lk {

static constexpr int HUB_CHUNK = LK_HUB_CHUNK;  // row entries per insert work item
static constexpr int HUB_SCAN_CHUNK = 4096; // table slots per scan work item

template <typename WT>
__device__ __forceinline__ bool hub_eligible(const MoveArgs<WT> &a, int32_t i, bool refine) {
  if (!refine) {
    if (a.processed[i]) return false;
    a.processed[i] = 1;
    return a.in_range ? a.in_range[i] != 0 : true;
  }
  return a.changed[a.CB[i]] && a.C[i] == i && a.Sig[i] == a.K[i];
}

// Single block: hub k of the list gets its table offset toff[k], size tsz[k]
// (0 when not eligible), insert-work offset ioff[k] and scan-work offset
// soff[k]; the totals go to hw.tot[0..2].
template <typename WT>
__global__ void __launch_bounds__(1024) hub_prep_k(MoveArgs<WT> a, bool refine, HubWork hw, int64_t cluster_cap) {
  __shared__ int64_t warp_s[3][32];
  __shared__ int64_t carry[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t base = 0; base < a.list_n; base += blockDim.x) {
    const int64_t k = base + threadIdx.x;
    int64_t v[3] = {0, 0, 0};
    if (k < a.list_n) {
      const int32_t i = a.list[k];
      int64_t tsz = 0;
      if (hub_eligible(a, i, refine)) {
        const int64_t deg = a.g.off[i + 1] - a.g.off[i];
        const int64_t cap = deg < a.g.n ? deg : a.g.n;
        if (cap <= cluster_cap) {
          tsz = -1;  // decided by a cluster with the table in distributed shared memory
        } else {
          // at least twice the distinct keys, in whole scan chunks (the home
          // slot comes from a multiply-shift, so any size works)
          const int64_t t = ((2 * cap + HUB_SCAN_CHUNK - 1) / HUB_SCAN_CHUNK) * HUB_SCAN_CHUNK;
          v[0] = t;
          v[1] = (deg + HUB_CHUNK - 1) / HUB_CHUNK;
          v[2] = t / HUB_SCAN_CHUNK;
          tsz = t;
        }
      }
      hw.tsz[k] = tsz;
    }
    // block-wide exclusive scans of the three counts
    int64_t incl[3];
    for (int q = 0; q < 3; q++) {
      int64_t x = v[q];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = shfl_i64(x, (lane - o) & 31);
        if (lane >= o) x += y;
      }
      incl[q] = x;
      if (lane == 31) warp_s[q][warp] = x;
    }
    __syncthreads();
    if (k < a.list_n) {
      int64_t *outs[3] = {hw.toff, hw.ioff, hw.soff};
      for (int q = 0; q < 3; q++) {
        int64_t pre = carry[q];
        for (int w = 0; w < warp; w++) pre += warp_s[q][w];
        outs[q][k] = pre + incl[q] - v[q];
      }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      int64_t s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += warp_s[threadIdx.x][w];
      carry[threadIdx.x] += s;
    }
    __syncthreads();
  }
  if (threadIdx.x < 3) {
    hw.tot[threadIdx.x] = carry[threadIdx.x];
    int64_t *outs[3] = {hw.toff, hw.ioff, hw.soff};
    outs[threadIdx.x][a.list_n] = carry[threadIdx.x];
  }
}

// last k with offs[k] <= w, over k in [0, n)
__device__ __forceinline__ int64_t find_item(const int64_t *offs, int64_t n, int64_t w) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Insert of one (community, weight) into a hub's global table, starting with
// the compare-and-swap of the home slot (one round trip for a new key or a
// key already there; the probe sequence only after a collision).
template <typename VT>
__device__ __forceinline__ void hub_table_add_cas(int32_t *keys, VT *vals, uint64_t t, int32_t c, u64 w,
                                                  u64 *err) {
  uint64_t s = ((uint64_t)hash32(c) * t) >> 32;
  for (uint64_t probe = 0; probe < t; probe++) {
    const int32_t old = atomicCAS(&keys[s], LEIDEN_EMPTY_KEY, c);
    if (old == LEIDEN_EMPTY_KEY || old == c) { add_val(&vals[s], w); return; }
    s = s + 1 == t ? 0 : s + 1;
  }
  atomicOr(err, 16ull);
}

// With 32-bit table values (the 64-bit score path) a slot is one 64-bit word
// of the value scratch: the key + 1 in its low half (0: empty, which is how
// the scratch is left), the summed weight in its high half, so the
// compare-and-swap of the key and the add of the weight touch the same DRAM
// sector, and the drain reads one array instead of two.
__device__ __forceinline__ void hub_table_add_packed(u64 *tab, uint64_t t, int32_t c, u64 w, u64 *err) {
  const uint32_t key = (uint32_t)c + 1u;
  uint64_t s = ((uint64_t)hash32(c) * t) >> 32;
  for (uint64_t probe = 0; probe < t; probe++) {
    uint32_t *slot = reinterpret_cast<uint32_t *>(&tab[s]);   // [0] key + 1, [1] weight
    const uint32_t old = atomicCAS(slot, 0u, key);
    if (old == 0u || old == key) { atomicAdd(slot + 1, (uint32_t)w); return; }
    s = s + 1 == t ? 0 : s + 1;
  }
  atomicOr(err, 16ull);
}

template <typename WT, typename VT>
__global__ void __launch_bounds__(256) hub_insert_k(MoveArgs<WT> a, bool refine, HubWork hw) {
  constexpr bool PACKED = sizeof(VT) == 4;
  constexpr int U = LK_HUB_UNROLL;
  __shared__ u64 wscratch[8][32];
  const int64_t nitems = hw.tot[1];
  for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int64_t k = find_item(hw.ioff, a.list_n, w);
    const int32_t i = a.list[k];
    const int64_t e0 = a.g.off[i], e1 = a.g.off[i + 1];
    const int64_t c0 = e0 + (w - hw.ioff[k]) * HUB_CHUNK;
    const int64_t c1 = c0 + HUB_CHUNK < e1 ? c0 + HUB_CHUNK : e1;
    const int64_t t = hw.tsz[k];
    int32_t *keys = a.gkeys + hw.toff[k];
    VT *vals = reinterpret_cast<VT *>(a.gvals) + hw.toff[k];
    const int32_t cbi = refine ? a.CB[i] : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // U warp-uniform 32-entry chunks per step, blockDim.x apart
    for (int64_t cb = c0 + 32 * warp; cb < c1; cb += (int64_t)blockDim.x * U) {
      int32_t cc[U];
      u64 wv[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int64_t e = cb + (int64_t)u * blockDim.x + lane;
        int32_t j = -1;
        wv[u] = 0;
        if (e < c1) {
          j = a.g.idx[e];
          wv[u] = (u64)(int64_t)a.g.w[e];
          if (j == i) j = -1;
          else if ((uint32_t)j >= (uint32_t)a.g.n) { atomicOr(&a.ctr[CTR_ERROR], 64ull); j = -1; }
        }
        cc[u] = j;
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int32_t j = cc[u];
        bool ok = j >= 0;
        if (refine && ok && a.CB[j] != cbi) ok = false;
        cc[u] = ok ? a.C[j] : LEIDEN_EMPTY_KEY;
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        u64 sum = 0;
        if (warp_combine((unsigned long long)(uint32_t)cc[u], cc[u] != LEIDEN_EMPTY_KEY, wv[u], &sum,
                         wscratch[warp]))
          wv[u] = sum;
        else
          cc[u] = LEIDEN_EMPTY_KEY;
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (cc[u] == LEIDEN_EMPTY_KEY) continue;
        if (PACKED) hub_table_add_packed(a.gvals + hw.toff[k], (uint64_t)t, cc[u], wv[u], &a.ctr[CTR_ERROR]);
        else hub_table_add_cas(keys, vals, (uint64_t)t, cc[u], wv[u], &a.ctr[CTR_ERROR]);
      }
    }
  }
}

template <typename WT, typename ST>
__device__ __forceinline__ bool hub_better(ST sc, int32_t c, ST bsc, int32_t bc) {
  return c != INT32_MAX && (bc == INT32_MAX || sc > bsc || (sc == bsc && c < bc));
}

template <typename WT, typename ST>
__global__ void __launch_bounds__(256) hub_scan_k(MoveArgs<WT> a, HubWork hw) {
  __shared__ ST r_sc[8];
  __shared__ int32_t r_c[8];
  __shared__ int64_t r_kid[8];
  __shared__ int64_t r_cand[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nitems = hw.tot[2];
  for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int64_t k = find_item(hw.soff, a.list_n, w);
    const int32_t i = a.list[k];
    const int32_t d = a.C[i];
    const ST A = (ST)a.A;
    const ST B = (ST)a.p * (ST)a.K[i];
    const int64_t s0 = (w - hw.soff[k]) * HUB_SCAN_CHUNK;
    int32_t *keys = a.gkeys + hw.toff[k];
    typename TableVal<ST>::type *vals = reinterpret_cast<typename TableVal<ST>::type *>(a.gvals) + hw.toff[k];
    ST bsc = 0;
    int32_t bc = INT32_MAX;
    int64_t kid = 0, cand = 0;
    constexpr bool PACKED = sizeof(typename TableVal<ST>::type) == 4;
    u64 *tab = a.gvals + hw.toff[k];
    for (int64_t s = s0 + threadIdx.x; s < s0 + HUB_SCAN_CHUNK; s += blockDim.x) {
      int32_t c;
      int64_t v;
      if (PACKED) {
        const u64 x = tab[s];
        if (x == 0) continue;
        c = (int32_t)((uint32_t)x - 1u);
        v = (int64_t)(x >> 32);
        tab[s] = 0;                  // reset for the next user of the scratch
      } else {
        c = keys[s];
        if (c == LEIDEN_EMPTY_KEY) continue;
        v = (int64_t)vals[s];
        keys[s] = LEIDEN_EMPTY_KEY;  // reset for the next user of the scratch
        vals[s] = 0;
      }
      cand++;
      if (c == d) { kid = v; continue; }
      const ST sc = A * (ST)v - B * (ST)sigma_for_score(a.Sig, c);
      if (hub_better<WT, ST>(sc, c, bsc, bc)) { bsc = sc; bc = c; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const ST osc = shfl_xor_any<ST>(bsc, o);
      const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
      kid += shfl_xor_i64(kid, o);
      cand += shfl_xor_i64(cand, o);
      if (hub_better<WT, ST>(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
    }
    if (lane == 0) { r_sc[warp] = bsc; r_c[warp] = bc; r_kid[warp] = kid; r_cand[warp] = cand; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < (int)(blockDim.x >> 5); q++) {
        kid += r_kid[q];
        cand += r_cand[q];
        if (hub_better<WT, ST>(r_sc[q], r_c[q], bsc, bc)) { bsc = r_sc[q]; bc = r_c[q]; }
      }
      hw.psc[w] = (i128)bsc;
      hw.pc[w] = bc;
      hw.pkid[w] = kid;
      if (cand) atomicAdd(&a.ctr[CTR_CANDIDATES], (u64)cand);
    }
    __syncthreads();
  }
}

template <typename WT, typename ST, bool REFINE, bool ASYNC>
__global__ void __launch_bounds__(256) hub_final_k(MoveArgs<WT> a, HubWork hw) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.list_n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (hw.tsz[k] <= 0) continue;  // not eligible, or decided by a cluster
    const int32_t i = a.list[k];
    const int32_t d = a.C[i];
    i128 bsc = 0;
    int32_t bc = INT32_MAX;
    int64_t kid = 0;
    for (int64_t w = hw.soff[k]; w < hw.soff[k + 1]; w++) {
      kid += hw.pkid[w];
      if (hub_better<WT, i128>(hw.psc[w], hw.pc[w], bsc, bc)) { bsc = hw.psc[w]; bc = hw.pc[w]; }
    }
    const int64_t Ki = a.K[i];
    atomicAdd(&a.ctr[CTR_SCANNED_ENTRIES], (u64)(a.g.off[i + 1] - a.g.off[i]));
    atomicAdd(&a.ctr[CTR_SCANNED_VERTICES], 1ull);
    if (bc == INT32_MAX) continue;
    const i128 S = bsc - (i128)a.A * kid - (i128)a.p * Ki * (Ki - a.Sig[d]);
    if (S <= 0) continue;
    if (REFINE && a.C[bc] != bc) continue;
    if (ASYNC) {
      bool ok;
      if (!REFINE) {
        if (a.Sig[d] == Ki && a.Sig[bc] == a.K[bc] && bc > d) continue;  // minimum-label rule
        atomic_add_i64(&a.Sig[d], -Ki);
        atomic_add_i64(&a.Sig[bc], Ki);
        a.C[i] = bc;
        if (a.dynamic) { a.changed[d] = 1; a.changed[bc] = 1; }
        ok = true;
        // its neighbours are re-marked by the big-row marking kernel
        const u64 slot = atomicAdd(&a.ctr[CTR_BIG], 1ull);
        a.big[slot] = i;
      } else {
        ok = refine_join_async(a.Sig, i, Ki, bc);
        if (ok) a.C[i] = bc;
      }
      if (ok) {
        atomicAdd(&a.ctr[CTR_MOVES], 1ull);
        atomic_add_i128(&a.ctr[CTR_SUMS_LO], S);
      }
    } else {
      const u64 slot = atomicAdd(a.prop_count, 1ull);
      a.prop_i[slot] = i;
      a.prop_c[slot] = bc;
      a.prop_S[slot] = S;
      if (REFINE) a.stamp[i] = a.stamp_val;
    }
  }
}

// ---------------------------------------------------------------------------
// Cluster path: one thread-block cluster of HC_CTAS CTAs decides one hub at a
// time, its hashtable spread over the CTAs' shared memory (distributed shared
// memory, HC_SLOTS slots per CTA; slot s lives in CTA s / HC_SLOTS).  The
// CTAs split the row, combine equal communities per warp and insert into the
// owning CTA's slice with shared-memory atomics across the cluster; after a
// cluster barrier each CTA scans its own slice, and CTA 0 reduces the slices'
// bests and takes the decision (Eq. 2 scaled, the move rule) -- one kernel
// instead of the insert / scan / final chain through global memory, for hubs
// with at most HC_CTAS * HC_SLOTS / 2 distinct candidates.
// ---------------------------------------------------------------------------
static constexpr int HC_CTAS = 8;
static constexpr int HC_LOG2 = 14;
static constexpr uint32_t HC_SLOTS = 1u << HC_LOG2;
static constexpr int HC_THREADS = 512;

template <typename WT, typename ST, bool REFINE, bool ASYNC>
__global__ void __launch_bounds__(HC_THREADS) hub_cluster_k(MoveArgs<WT> a, HubWork hw) {
  namespace cg = cooperative_groups;
  typedef typename TableVal<ST>::type VT;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  VT *vals = reinterpret_cast<VT *>(smem);
  int32_t *keys = reinterpret_cast<int32_t *>(vals + HC_SLOTS);
  __shared__ u64 wscratch[HC_THREADS / 32][32];
  __shared__ ST r_sc[HC_THREADS / 32];
  __shared__ int32_t r_c[HC_THREADS / 32];
  __shared__ int64_t r_kid[HC_THREADS / 32];
  __shared__ int64_t r_cand[HC_THREADS / 32];
  __shared__ ST p_sc;        // this CTA's best over its slice, read by CTA 0
  __shared__ int32_t p_c;
  __shared__ int64_t p_kid;
  const unsigned rank = cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cid = blockIdx.x / HC_CTAS, ncl = gridDim.x / HC_CTAS;
  for (int64_t k = cid; k < a.list_n; k += ncl) {   // the same k in every CTA of the cluster
    if (hw.tsz[k] >= 0) continue;                    // not eligible, or on the global path
    const int32_t i = a.list[k];
    const int64_t e0 = a.g.off[i], e1 = a.g.off[i + 1];
    // the hub's table: at least twice its distinct candidates, a power of two
    // of slots per CTA (at most HC_SLOTS); clearing and scanning cost its size
    const int64_t cap = (e1 - e0) < a.g.n ? (e1 - e0) : a.g.n;
    int lg = 8;
    while (lg < HC_LOG2 && ((int64_t)HC_CTAS << lg) < 2 * cap) lg++;
    const uint32_t LS = 1u << lg;                    // slots per CTA for this hub
    const uint64_t TT = (uint64_t)LS * HC_CTAS;
    for (uint32_t sl = threadIdx.x; sl < LS; sl += blockDim.x) { keys[sl] = LEIDEN_EMPTY_KEY; vals[sl] = 0; }
    cl.sync();
    const int32_t cbi = REFINE ? a.CB[i] : 0;
    const int64_t stride = (int64_t)HC_CTAS * blockDim.x;
    for (int64_t base = e0 + (int64_t)rank * blockDim.x + warp * 32; base < e1; base += stride) {
      const int64_t e = base + lane;
      int32_t c = LEIDEN_EMPTY_KEY;
      u64 wv = 0;
      if (e < e1) {
        const int32_t j = a.g.idx[e];
        bool ok = j != i;
        if (ok && (uint32_t)j >= (uint32_t)a.g.n) { atomicOr(&a.ctr[CTR_ERROR], 64ull); ok = false; }
        if (REFINE && ok && a.CB[j] != cbi) ok = false;
        if (ok) { c = a.C[j]; wv = (u64)(int64_t)a.g.w[e]; }
      }
      u64 sum = 0;
      if (warp_combine((unsigned long long)(uint32_t)c, c != LEIDEN_EMPTY_KEY, wv, &sum, wscratch[warp])) {
        uint64_t sl = ((uint64_t)hash32(c) * TT) >> 32;
        bool done = false;
        for (uint64_t probe = 0; probe < TT && !done; probe++) {
          const unsigned owner = (unsigned)(sl >> lg);
          const uint32_t loc = (uint32_t)(sl & (LS - 1));
          int32_t *kp = cl.map_shared_rank(keys, owner) + loc;
          VT *vp = cl.map_shared_rank(vals, owner) + loc;
          const int32_t kk = *(volatile int32_t *)kp;
          if (kk == c) { add_val(vp, sum); done = true; break; }
          if (kk == LEIDEN_EMPTY_KEY) {
            const int32_t old = atomicCAS(kp, LEIDEN_EMPTY_KEY, c);
            if (old == LEIDEN_EMPTY_KEY || old == c) { add_val(vp, sum); done = true; break; }
          }
          sl = sl + 1 == TT ? 0 : sl + 1;
        }
        if (!done) atomicOr(&a.ctr[CTR_ERROR], 16ull);
      }
    }
    cl.sync();
    // this CTA's slice: best candidate and the weight towards the own community
    const int32_t d = a.C[i];
    const int64_t Ki = a.K[i];
    const ST A = (ST)a.A, B = (ST)a.p * (ST)Ki;
    ST bsc = 0;
    int32_t bc = INT32_MAX;
    int64_t kid = 0, cand = 0;
    for (uint32_t sl = threadIdx.x; sl < LS; sl += blockDim.x) {
      const int32_t c = keys[sl];
      if (c == LEIDEN_EMPTY_KEY) continue;
      const int64_t v = (int64_t)vals[sl];
      cand++;
      if (c == d) { kid = v; continue; }
      const ST sc = A * (ST)v - B * (ST)sigma_for_score(a.Sig, c);
      if (hub_better<WT, ST>(sc, c, bsc, bc)) { bsc = sc; bc = c; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const ST osc = shfl_xor_any<ST>(bsc, o);
      const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
      kid += shfl_xor_i64(kid, o);
      cand += shfl_xor_i64(cand, o);
      if (hub_better<WT, ST>(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
    }
    if (lane == 0) { r_sc[warp] = bsc; r_c[warp] = bc; r_kid[warp] = kid; r_cand[warp] = cand; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < (int)(blockDim.x >> 5); q++) {
        kid += r_kid[q];
        cand += r_cand[q];
        if (hub_better<WT, ST>(r_sc[q], r_c[q], bsc, bc)) { bsc = r_sc[q]; bc = r_c[q]; }
      }
      p_sc = bsc;
      p_c = bc;
      p_kid = kid;
      if (cand) atomicAdd(&a.ctr[CTR_CANDIDATES], (u64)cand);
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
      for (unsigned r = 1; r < HC_CTAS; r++) {
        const ST osc = *cl.map_shared_rank(&p_sc, r);
        const int32_t oc = *cl.map_shared_rank(&p_c, r);
        kid += *cl.map_shared_rank(&p_kid, r);
        if (hub_better<WT, ST>(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
      }
      atomicAdd(&a.ctr[CTR_SCANNED_ENTRIES], (u64)(e1 - e0));
      atomicAdd(&a.ctr[CTR_SCANNED_VERTICES], 1ull);
      bool go = bc != INT32_MAX;
      i128 S = 0;
      if (go) {
        S = (i128)bsc - (i128)a.A * kid - (i128)a.p * Ki * (Ki - a.Sig[d]);
        go = S > 0;
        if (REFINE && go && a.C[bc] != bc) go = false;
      }
      if (go && ASYNC) {
        bool ok;
        if (!REFINE) {
          ok = !(a.Sig[d] == Ki && a.Sig[bc] == a.K[bc] && bc > d);  // minimum-label rule
          if (ok) {
            atomic_add_i64(&a.Sig[d], -Ki);
            atomic_add_i64(&a.Sig[bc], Ki);
            a.C[i] = bc;
            if (a.dynamic) { a.changed[d] = 1; a.changed[bc] = 1; }
            const u64 slot = atomicAdd(&a.ctr[CTR_BIG], 1ull);  // neighbours re-marked by the big-row kernel
            a.big[slot] = i;
          }
        } else {
          ok = refine_join_async(a.Sig, i, Ki, bc);
          if (ok) a.C[i] = bc;
        }
        if (ok) {
          atomicAdd(&a.ctr[CTR_MOVES], 1ull);
          atomic_add_i128(&a.ctr[CTR_SUMS_LO], S);
        }
      } else if (go) {
        const u64 slot = atomicAdd(a.prop_count, 1ull);
        a.prop_i[slot] = i;
        a.prop_c[slot] = bc;
        a.prop_S[slot] = S;
        if (REFINE) a.stamp[i] = a.stamp_val;
      }
    }
    cl.sync();   // CTA 0 has read every slice's best before the next hub reuses them
  }
}

// Clusters resident at once for the cluster path (0: not available), per
// instantiation, queried once.
template <typename WT, typename ST, bool REFINE, bool ASYNC>
static int hub_clusters() {
  static int n = -1;
  if (n >= 0) return n;
  auto k = hub_cluster_k<WT, ST, REFINE, ASYNC>;
  const size_t smem = (size_t)HC_SLOTS * (sizeof(typename TableVal<ST>::type) + sizeof(int32_t));
  n = 0;
  if (cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return n;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(HC_CTAS, 1, 1);
  cfg.blockDim = dim3(HC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr{};
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = HC_CTAS;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int c = 0;
  if (cudaOccupancyMaxActiveClusters(&c, (const void *)k, &cfg) != cudaSuccess) {
    cudaGetLastError();
    c = 0;
  }
  n = c;
  return n;
}

// Re-marks the neighbours of long movers as unprocessed: every block walks
// every listed row, so one long row is spread over the whole grid.
__global__ void __launch_bounds__(256) mark_big_rows_k(const int32_t *big, const u64 *count, const int64_t *off,
                                                       const int32_t *idx, uint8_t *processed) {
  // bpr blocks per row: the whole grid on one row when there are few rows,
  // one block per row (rows strided over the grid) when there are many
  const u64 nb = *count;
  if (nb == 0) return;
  const u64 bpr = gridDim.x / nb > 0 ? gridDim.x / nb : 1;
  const u64 rows_at_once = gridDim.x / bpr;
  const u64 part = blockIdx.x % bpr;
  for (u64 m = blockIdx.x / bpr; m < nb && blockIdx.x < rows_at_once * bpr; m += rows_at_once) {
    const int32_t i = big[m];
    const int64_t e0 = off[i], e1 = off[i + 1];
    const int64_t step = (int64_t)bpr * blockDim.x;
    for (int64_t e = e0 + (int64_t)part * blockDim.x + threadIdx.x; e < e1; e += 4 * step) {
      int32_t j[4];
#pragma unroll
      for (int u = 0; u < 4; u++) j[u] = e + u * step < e1 ? idx[e + u * step] : -1;
      uint8_t f[4];   // read before the store, as in the apply
#pragma unroll
      for (int u = 0; u < 4; u++) f[u] = j[u] >= 0 ? processed[j[u]] : 0;
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (f[u]) processed[j[u]] = 0;
    }
  }
}

void launch_mark_big(const int32_t *big, const u64 *count, const int64_t *off, const int32_t *idx,
                     uint8_t *processed, int sms, cudaStream_t s) {
  LK_COUNTED mark_big_rows_k<<<sms * 4, 256, 0, s>>>(big, count, off, idx, processed);
}

template <typename WT, typename ST, bool REFINE, bool ASYNC>
void launch_hubs(const MoveArgs<WT> &a, const HubWork &hw, int sms, cudaStream_t s) {
  if (a.list_n <= 0) return;
  const int ncl = LK_HUB_CLUSTERS ? hub_clusters<WT, ST, REFINE, ASYNC>() : 0;
  const int64_t cluster_cap = ncl > 0 ? (int64_t)HC_CTAS * HC_SLOTS / 2 : 0;
  LK_COUNTED hub_prep_k<WT><<<1, 1024, 0, s>>>(a, REFINE, hw, cluster_cap);
  if (ncl > 0) {
    int64_t nc = std::min<int64_t>(ncl, a.list_n);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(nc * HC_CTAS), 1, 1);
    cfg.blockDim = dim3(HC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)HC_SLOTS * (sizeof(typename TableVal<ST>::type) + sizeof(int32_t));
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = HC_CTAS;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    note_launch();
    cudaLaunchKernelEx(&cfg, hub_cluster_k<WT, ST, REFINE, ASYNC>, a, hw);
  }
  // grid-stride over equal work items: exactly the resident blocks
  auto ins = hub_insert_k<WT, typename TableVal<ST>::type>;
  auto scn = hub_scan_k<WT, ST>;
  LK_COUNTED ins<<<(unsigned)resident_blocks((const void *)ins, 256, 0, sms), 256, 0, s>>>(a, REFINE, hw);
  LK_COUNTED scn<<<(unsigned)resident_blocks((const void *)scn, 256, 0, sms), 256, 0, s>>>(a, hw);
  LK_COUNTED hub_final_k<WT, ST, REFINE, ASYNC><<<(unsigned)((a.list_n + 255) / 256), 256, 0, s>>>(a, hw);
}

#define LK_HUB_INST(WT, ST)                                                                              \
  template void launch_hubs<WT, ST, false, false>(const MoveArgs<WT> &, const HubWork &, int, cudaStream_t); \
  template void launch_hubs<WT, ST, true, false>(const MoveArgs<WT> &, const HubWork &, int, cudaStream_t);  \
  template void launch_hubs<WT, ST, false, true>(const MoveArgs<WT> &, const HubWork &, int, cudaStream_t);  \
  template void launch_hubs<WT, ST, true, true>(const MoveArgs<WT> &, const HubWork &, int, cudaStream_t);
LK_HUB_INST(int32_t, int64_t)
LK_HUB_INST(int32_t, i128)
LK_HUB_INST(int64_t, int64_t)
LK_HUB_INST(int64_t, i128)
#undef LK_HUB_INST

}  // namespace lk
