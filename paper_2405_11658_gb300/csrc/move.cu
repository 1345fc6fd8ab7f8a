// move.cu -- local-moving (Alg. leidenlm) and refinement (Alg. leidenre)
// kernels for sm_103a.
//
// Every vertex of a (colour class, degree tier) bucket gets a group of lanes,
// a block, or a block with a global-memory table (hub rows).  The group hashes
// K_{i->c} = sum of w_ij over neighbours j != i with C'[j] = c into an
// open-addressing table (scanCommunities / scanBounded), then takes the argmax
// of the scaled delta-modularity of Eq. 2 over the table's keys other than its
// own community d (ties to the smallest ID).  All sums are integers, so the
// result does not depend on hashing order or thread timing.
//
// DET: decide kernels read a snapshot (nothing they read is written until the
// sub-sweep's apply kernel runs) and append proposals; apply kernels commit
// them.  ASYNC: the deciding group commits immediately with atomics, like the
// paper's asynchronous CPU implementation (Sec. 4.7), with the minimum-label
// rule for moves between singleton communities.
#include <limits.h>

#include "common.cuh"
#include "internal.h"

namespace lk {

template <typename ST>
__device__ __forceinline__ bool better(ST sc, int32_t c, ST bsc, int32_t bc) {
  return c != INT32_MAX && (bc == INT32_MAX || sc > bsc || (sc == bsc && c < bc));
}

// Insert (c, w) into an open-addressing table of 2^log2H slots; the table has
// at least twice as many slots as the row has entries, so it never fills.
// Probing is bounded all the same: a full table sets *err and drops the entry.
template <typename VT>
__device__ __forceinline__ void table_add(int32_t *keys, VT *vals, int log2H, int32_t c, u64 w, u64 *err) {
  const uint32_t mask = (1u << log2H) - 1u;
  uint32_t s = hash32(c) >> (32 - log2H);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    int32_t k = *(volatile int32_t *)&keys[s];
    if (k == c) { add_val(&vals[s], w); return; }
    if (k == LEIDEN_EMPTY_KEY) {
      int32_t old = atomicCAS(&keys[s], LEIDEN_EMPTY_KEY, c);
      if (old == LEIDEN_EMPTY_KEY || old == c) { add_val(&vals[s], w); return; }
    }
    s = (s + 1) & mask;
  }
  atomicOr(err, 16ull);
}

// Scans table slots s0, s0 + step, ... < H of one vertex: candidate scores
// for every occupied slot other than the own community d, and the weight to
// d.  SCAN_UNROLL slots per lane are loaded first and their Sigma'[c] gathers
// issued together, so the gathers overlap instead of running back to back.
static constexpr int SCAN_UNROLL = LK_SCAN_UNROLL;
static constexpr int ROW_UNROLL = LK_ROW_UNROLL;  // row entries per lane in flight in the group kernels
static constexpr int BLOCK_ROW_UNROLL = LK_BLOCK_ROW_UNROLL;  // ... and in the block kernels
// Vertices per SM below which a whole-warp group tier runs as 4-warp blocks.
static constexpr int64_t SMALL_WAVE_VERTICES = 16;
template <typename ST, typename VT>
__device__ __forceinline__ void scan_slots(const int32_t *keys, const VT *vals, int H, int s0, int step,
                                           int32_t d, ST A, ST B, const int64_t *Sig, ST &bsc, int32_t &bc,
                                           int64_t &kid, int64_t &ncand) {
  for (int sb = s0; sb < H; sb += step * SCAN_UNROLL) {
    int32_t ck[SCAN_UNROLL];
    int64_t vk[SCAN_UNROLL], sg[SCAN_UNROLL];
#pragma unroll
    for (int u = 0; u < SCAN_UNROLL; u++) {
      const int sl = sb + u * step;
      ck[u] = sl < H ? keys[sl] : LEIDEN_EMPTY_KEY;
      vk[u] = ck[u] != LEIDEN_EMPTY_KEY ? (int64_t)vals[sl] : 0;
    }
#pragma unroll
    for (int u = 0; u < SCAN_UNROLL; u++)
      sg[u] = (ck[u] != LEIDEN_EMPTY_KEY && ck[u] != d) ? sigma_for_score(Sig, ck[u]) : 0;
#pragma unroll
    for (int u = 0; u < SCAN_UNROLL; u++) {
      const int32_t c = ck[u];
      if (c == LEIDEN_EMPTY_KEY) continue;
      ncand++;
      if (c == d) { kid = vk[u]; continue; }
      const ST sc = A * (ST)vk[u] - B * (ST)sg[u];
      if (better(sc, c, bsc, bc)) { bsc = sc; bc = c; }
    }
  }
}

// Vertex pruning: neighbour j of a mover is unprocessed again.  Most such
// neighbours already are (an earlier mover re-marked them): reading the flag
// first spares the random byte store.
__device__ __forceinline__ void unmark(uint8_t *processed, int32_t j) {
  if (processed[j]) processed[j] = 0;
}

// Eligibility of vertex i, decided by one thread.
template <bool REFINE, typename WT>
__device__ __forceinline__ bool eligible(const MoveArgs<WT> &a, int32_t i) {
  if (!REFINE) {
    if (a.processed[i]) return false;
    a.processed[i] = 1;                                  // prune
    return a.in_range ? a.in_range[i] != 0 : true;       // inAffectedRange
  } else {
    // reading: the flag of i's bound; i is still isolated iff Sigma'[i] = K'[i]
    return a.changed[a.CB[i]] && a.C[i] == i && a.Sig[i] == a.K[i];
  }
}

// Commit of an ASYNC move by one thread (the paper's in-place update).
template <bool REFINE, typename WT>
__device__ __forceinline__ bool commit_async(const MoveArgs<WT> &a, int32_t i, int32_t d,
                                             int32_t c) {
  const int64_t Ki = a.K[i];
  if (!REFINE) {
    // minimum-label rule for moves between singletons (Lu, Halappanavar and
    // Kalyanaraman 2015): two singletons deciding at the same time would swap
    // into each other's community; a singleton joins another singleton only
    // if that one has the smaller label
    if (a.Sig[d] == Ki && a.Sig[c] == a.K[c] && c > d) return false;
    atomic_add_i64(&a.Sig[d], -Ki);
    atomic_add_i64(&a.Sig[c], Ki);
    a.C[i] = c;
    if (a.dynamic) { a.changed[d] = 1; a.changed[c] = 1; }
    return true;
  } else {
    if (!refine_join_async(a.Sig, i, Ki, c)) return false;
    a.C[i] = c;
    return true;
  }
}

// ---------------------------------------------------------------------------
// Group tier: G lanes and 2^LOG2H shared slots per vertex.
// ---------------------------------------------------------------------------
#if LK_GROUP_MINB > 0
#define LK_GROUP_BOUNDS __launch_bounds__(256, LK_GROUP_MINB)
#else
#define LK_GROUP_BOUNDS
#endif
template <int G, int LOG2H, bool REFINE, bool ASYNC, typename WT, typename ST>
__global__ void LK_GROUP_BOUNDS decide_group(MoveArgs<WT> a) {
  constexpr int H = 1 << LOG2H;
  constexpr int GPW = 32 / G;
  extern __shared__ __align__(16) unsigned char smem[];
  const int wpb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = lane / G, gl = lane % G;
  const int leader = gw * G;
  typedef typename TableVal<ST>::type VT;
  VT *vals = reinterpret_cast<VT *>(smem) + (size_t)(warp * GPW + gw) * H;
  int32_t *keys = reinterpret_cast<int32_t *>(reinterpret_cast<VT *>(smem) + (size_t)wpb * GPW * H) +
                  (size_t)(warp * GPW + gw) * H;
  __shared__ u64 wscratch[8][32];  // blocks of at most 256 threads
  u64 *wscr = wscratch[warp];

  int64_t scanned = 0, nvert = 0, ncand = 0, nmoves = 0;
  i128 accS = 0;
  const int64_t wglob = (int64_t)blockIdx.x * wpb + warp;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  for (int64_t wb = wglob * GPW; wb < a.list_n; wb += nw * GPW) {
    const int64_t li = wb + gw;
    const bool valid = li < a.list_n;
    const int32_t i = valid ? a.list[li] : 0;
    // The row bounds, C'[i], K'[i] and (DET, a read-only snapshot) Sigma'[d]
    // do not depend on the eligibility test.  Where most listed vertices are
    // eligible they are loaded alongside it (one round of loads instead of a
    // chain); elsewhere only for the vertices that pass it.
    int64_t h0 = 0, h1 = 0, Ki = 0, hSd = 0;
    int32_t hd = 0;
    if (a.spec) {
      h0 = a.g.off[i];
      h1 = a.g.off[i + 1];
      hd = a.C[i];
      Ki = a.K[i];
      if (!ASYNC) hSd = a.Sig[hd];
    }
    bool act = false;
    if (gl == 0 && valid) act = eligible<REFINE>(a, i);
    act = __shfl_sync(FULL_MASK, act, leader);
    if (!a.spec && act) {
      h0 = a.g.off[i];
      h1 = a.g.off[i + 1];
      hd = a.C[i];
      Ki = a.K[i];
      if (!ASYNC) hSd = a.Sig[hd];
    }
    int32_t d = 0;
    int64_t e0 = 0, e1 = 0;
    int lh = 1;  // table sized for this row: 2^lh >= 2 * degree, lh <= LOG2H
    if (act) {
      e0 = h0;
      e1 = h1;
      while (lh < LOG2H && ((int64_t)1 << lh) < 2 * (e1 - e0)) lh++;
    }
    // the longest row of the warp's groups; every loop below is warp-uniform
    // so the lanes can combine equal (group, community) keys
    int64_t span = act ? e1 - e0 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int64_t y = shfl_xor_i64(span, o);
      span = y > span ? y : span;
    }
    // rows of at most G entries: one entry per lane, and the combine alone
    // yields every distinct community with its summed weight -- no table
    const bool one_step = span <= G;
    if (act && !one_step)
      for (int s = gl; s < (1 << lh); s += G) { keys[s] = LEIDEN_EMPTY_KEY; vals[s] = 0; }
    __syncwarp();
    const int32_t cbi = (REFINE && act) ? a.CB[i] : 0;
    if (act) d = hd;
    ST bsc = 0;
    int32_t bc = INT32_MAX;
    int64_t kid = 0;
    if (one_step) {
      const int64_t e = e0 + gl;
      const bool in = act && e < e1;
      const int32_t j = in ? a.g.idx[e] : -1;
      const u64 wv = in ? (u64)(int64_t)a.g.w[e] : 0;
      bool ok = in && j != i;                            // self = false
      if (ok && (uint32_t)j >= (uint32_t)a.g.n) { atomicOr(&a.ctr[CTR_ERROR], 64ull); ok = false; }
      if (REFINE && ok && a.CB[j] != cbi) ok = false;    // scanBounded
      const int32_t c = ok ? a.C[j] : LEIDEN_EMPTY_KEY;
      u64 sum = 0;
      const unsigned long long key = ((unsigned long long)(uint32_t)gw << 32) | (uint32_t)c;
      if (warp_combine(key, ok, wv, &sum, wscr)) {
        ncand++;
        if (c == d) {
          kid = (int64_t)sum;
        } else {
          const ST sc = (ST)a.A * (ST)(int64_t)sum - (ST)a.p * (ST)Ki * (ST)sigma_for_score(a.Sig, c);
          bsc = sc;
          bc = c;
        }
      }
    } else {
      for (int64_t xb = 0; xb < span; xb += (int64_t)G * ROW_UNROLL) {
        // ROW_UNROLL entries per lane: all loads and gathers first, then the
        // warp-uniform combine and table updates
        int32_t cc[ROW_UNROLL];
        u64 wv[ROW_UNROLL];
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; u++) {
          const int64_t e = e0 + xb + (int64_t)u * G + gl;
          const bool in = act && e < e1;
          const int32_t j = in ? a.g.idx[e] : -1;
          wv[u] = in ? (u64)(int64_t)a.g.w[e] : 0;
          bool ok = in && j != i;                         // self = false
          if (ok && (uint32_t)j >= (uint32_t)a.g.n) { atomicOr(&a.ctr[CTR_ERROR], 64ull); ok = false; }
          cc[u] = ok ? j : -1;
        }
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; u++) {
          const int32_t j = cc[u];
          bool ok = j >= 0;
          if (REFINE && ok && a.CB[j] != cbi) ok = false;  // scanBounded
          cc[u] = ok ? a.C[j] : LEIDEN_EMPTY_KEY;
        }
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; u++) {
          u64 sum = 0;
          const unsigned long long key = ((unsigned long long)(uint32_t)gw << 32) | (uint32_t)cc[u];
          if (warp_combine(key, cc[u] != LEIDEN_EMPTY_KEY, wv[u], &sum, wscr))
            table_add(keys, vals, lh, cc[u], sum, &a.ctr[CTR_ERROR]);
        }
      }
      __syncwarp();
      if (act) {
        const ST A = (ST)a.A;
        const ST B = (ST)a.p * (ST)Ki;
        scan_slots<ST, VT>(keys, vals, 1 << lh, gl, G, d, A, B, a.Sig, bsc, bc, kid, ncand);
      }
    }
    if (act && gl == 0) { scanned += e1 - e0; nvert++; }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const ST osc = shfl_xor_any<ST>(bsc, o);
      const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
      kid += shfl_xor_i64(kid, o);
      if (better(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
    }
    bool propose = false;
    i128 S = 0;
    if (act && gl == 0 && bc != INT32_MAX) {
      S = (i128)bsc - (i128)a.A * kid - (i128)a.p * Ki * (Ki - (ASYNC ? a.Sig[d] : hSd));
      propose = S > 0;                                   // strictly better only
      if (REFINE && propose && a.C[bc] != bc) propose = false;  // target's vertex left
    }
    if (ASYNC) {
      if (propose) {
        propose = commit_async<REFINE>(a, i, d, bc);
        if (propose) { accS += S; nmoves++; }
      }
      if (!REFINE) {
        const bool mv = __shfl_sync(FULL_MASK, propose, leader);
        if (mv)
          for (int64_t e = e0 + gl; e < e1; e += G) unmark(a.processed, a.g.idx[e]);
      }
    } else {
      const u64 slot = warp_reserve(a.prop_count, propose);
      if (propose) {
        a.prop_i[slot] = i;
        a.prop_c[slot] = bc;
        a.prop_S[slot] = S;
        if (REFINE) a.stamp[i] = a.stamp_val;
      }
    }
    __syncwarp();
  }
  // counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    scanned += shfl_xor_i64(scanned, o);
    nvert += shfl_xor_i64(nvert, o);
    ncand += shfl_xor_i64(ncand, o);
    nmoves += shfl_xor_i64(nmoves, o);
    if (ASYNC) accS += shfl_xor_i128(accS, o);
  }
  if (lane == 0) {
    if (scanned) atomicAdd(&a.ctr[CTR_SCANNED_ENTRIES], (u64)scanned);
    if (nvert) atomicAdd(&a.ctr[CTR_SCANNED_VERTICES], (u64)nvert);
    if (ncand) atomicAdd(&a.ctr[CTR_CANDIDATES], (u64)ncand);
    if (ASYNC && nmoves) {
      atomicAdd(&a.ctr[CTR_MOVES], (u64)nmoves);
      atomic_add_i128(&a.ctr[CTR_SUMS_LO], accS);
    }
  }
}

// ---------------------------------------------------------------------------
// Thread tier: one lane per vertex, for rows of at most KMAX entries.  The
// row's neighbours, weights and communities are loaded into registers with
// all of the row's loads in flight at once, equal communities are merged in
// registers (the first occurrence keeps the sum), and the candidates' Sigma'
// are gathered together: no table, no cooperation between lanes, 32 vertices
// per warp instead of 32 / G.  The decision is the one of the other tiers
// (same scores, same tie-break).
// ---------------------------------------------------------------------------
template <int KMAX, bool REFINE, bool ASYNC, typename WT, typename ST>
__global__ void __launch_bounds__(256) decide_thread(MoveArgs<WT> a) {
  int64_t scanned = 0, nvert = 0, ncand = 0, nmoves = 0;
  i128 accS = 0;
  const int lane = threadIdx.x & 31;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform loop (the proposal reservation needs the whole warp)
  for (int64_t base = gt - lane; base < a.list_n; base += nt) {
    const int64_t li = base + lane;
    const bool valid = li < a.list_n;
    const int32_t i = valid ? a.list[li] : 0;
    int64_t e0 = 0, e1 = 0, Ki = 0, Sd = 0;
    int32_t d = 0;
    if (a.spec && valid) {
      e0 = a.g.off[i];
      e1 = a.g.off[i + 1];
      d = a.C[i];
      Ki = a.K[i];
      if (!ASYNC) Sd = a.Sig[d];
    }
    const bool act = valid && eligible<REFINE>(a, i);
    if (!a.spec && act) {
      e0 = a.g.off[i];
      e1 = a.g.off[i + 1];
      d = a.C[i];
      Ki = a.K[i];
      if (!ASYNC) Sd = a.Sig[d];
    }
    const int deg = act ? (int)(e1 - e0) : 0;  // at most KMAX by the tier
    const int32_t cbi = (REFINE && act) ? a.CB[i] : 0;
    int32_t cc[KMAX];
    int64_t ww[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
      cc[k] = k < deg ? a.g.idx[e0 + k] : -1;
      ww[k] = k < deg ? (int64_t)a.g.w[e0 + k] : 0;
    }
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
      const int32_t j = cc[k];
      bool ok = j >= 0 && j != i;                          // self = false
      if (ok && (uint32_t)j >= (uint32_t)a.g.n) { atomicOr(&a.ctr[CTR_ERROR], 64ull); ok = false; }
      if (REFINE && ok && a.CB[j] != cbi) ok = false;      // scanBounded
      cc[k] = ok ? a.C[j] : LEIDEN_EMPTY_KEY;
    }
    // merge equal communities into their first occurrence
#pragma unroll
    for (int k = 1; k < KMAX; k++) {
#pragma unroll
      for (int k2 = 0; k2 < k; k2++)
        if (cc[k] != LEIDEN_EMPTY_KEY && cc[k2] == cc[k]) {
          ww[k2] += ww[k];
          cc[k] = LEIDEN_EMPTY_KEY;
        }
    }
    int64_t sg[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; k++) sg[k] = (cc[k] != LEIDEN_EMPTY_KEY && cc[k] != d) ? sigma_for_score(a.Sig, cc[k]) : 0;
    const ST A = (ST)a.A;
    const ST B = (ST)a.p * (ST)Ki;
    ST bsc = 0;
    int32_t bc = INT32_MAX;
    int64_t kid = 0;
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
      const int32_t c = cc[k];
      if (c == LEIDEN_EMPTY_KEY) continue;
      ncand++;
      if (c == d) { kid = ww[k]; continue; }
      const ST sc = A * (ST)ww[k] - B * (ST)sg[k];
      if (better(sc, c, bsc, bc)) { bsc = sc; bc = c; }
    }
    if (act) { scanned += deg; nvert++; }
    bool propose = false;
    i128 S = 0;
    if (act && bc != INT32_MAX) {
      S = (i128)bsc - (i128)a.A * kid - (i128)a.p * Ki * (Ki - (ASYNC ? a.Sig[d] : Sd));
      propose = S > 0;                                     // strictly better only
      if (REFINE && propose && a.C[bc] != bc) propose = false;  // target's vertex left
    }
    if (ASYNC) {
      if (propose) {
        propose = commit_async<REFINE>(a, i, d, bc);
        if (propose) { accS += S; nmoves++; }
      }
      if (!REFINE && propose)
        for (int64_t e = e0; e < e1; e++) unmark(a.processed, a.g.idx[e]);
    } else {
      const u64 slot = warp_reserve(a.prop_count, propose);
      if (propose) {
        a.prop_i[slot] = i;
        a.prop_c[slot] = bc;
        a.prop_S[slot] = S;
        if (REFINE) a.stamp[i] = a.stamp_val;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    scanned += shfl_xor_i64(scanned, o);
    nvert += shfl_xor_i64(nvert, o);
    ncand += shfl_xor_i64(ncand, o);
    nmoves += shfl_xor_i64(nmoves, o);
    if (ASYNC) accS += shfl_xor_i128(accS, o);
  }
  if (lane == 0) {
    if (scanned) atomicAdd(&a.ctr[CTR_SCANNED_ENTRIES], (u64)scanned);
    if (nvert) atomicAdd(&a.ctr[CTR_SCANNED_VERTICES], (u64)nvert);
    if (ncand) atomicAdd(&a.ctr[CTR_CANDIDATES], (u64)ncand);
    if (ASYNC && nmoves) {
      atomicAdd(&a.ctr[CTR_MOVES], (u64)nmoves);
      atomic_add_i128(&a.ctr[CTR_SUMS_LO], accS);
    }
  }
}

// ---------------------------------------------------------------------------
// Block tiers: one block per vertex, table in shared memory.  The table is
// cleared once per block; each vertex lists the slots it occupies and the
// scan resets exactly those while reading them, so a vertex costs work in
// proportion to its row, not to the table size.
// ---------------------------------------------------------------------------
// Insert into a table; returns the slot if this call occupied it (else -1),
// so the caller can list the table's occupied slots.
template <typename VT>
__device__ __forceinline__ int table_add_new(int32_t *keys, VT *vals, int log2H, int32_t c, u64 w, u64 *err) {
  const uint32_t mask = (1u << log2H) - 1u;
  uint32_t s = hash32(c) >> (32 - log2H);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    int32_t k = *(volatile int32_t *)&keys[s];
    if (k == c) { add_val(&vals[s], w); return -1; }
    if (k == LEIDEN_EMPTY_KEY) {
      int32_t old = atomicCAS(&keys[s], LEIDEN_EMPTY_KEY, c);
      if (old == LEIDEN_EMPTY_KEY || old == c) {
        add_val(&vals[s], w);
        return old == LEIDEN_EMPTY_KEY ? (int)s : -1;
      }
    }
    s = (s + 1) & mask;
  }
  atomicOr(err, 16ull);
  return -1;
}

// Appends the slots the warp's lanes newly occupied to the used-slot list with
// one shared atomic per warp (a per-lane atomic on one counter serialises the
// whole block).  The whole warp must call.
__device__ __forceinline__ void list_new_slots(int slot, uint16_t *used, unsigned *nused) {
  const unsigned m = __ballot_sync(FULL_MASK, slot >= 0);
  if (!m) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(nused, (unsigned)__popc(m));
  base = __shfl_sync(FULL_MASK, base, leader);
  if (slot >= 0) used[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)slot;
}

// Block tier: one vertex at a time per block, its row spread over all warps.
// Warp 0 stages the headers of the block's next 32 listed vertices at once
// (eligibility, row bounds, C', K', Sigma'[d]) and keeps only the eligible
// ones, so neither a skipped vertex nor a header load costs the block a
// barrier or a round trip of its own.  A vertex takes two barriers: after the
// row's inserts, and after the used-slot scan; warp 0 then combines the
// warps' bests and proposes while the other warps start on the next row (the
// used-slot counter alternates between two words for that reason).
template <bool REFINE, bool ASYNC, typename WT, typename ST>
__global__ void __launch_bounds__(1024) decide_block(MoveArgs<WT> a, int log2H) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int32_t h_i[32], h_d[32];
  __shared__ int64_t h_e0[32], h_e1[32], h_K[32], h_Sd[32];
  __shared__ int32_t s_nact[2];
  __shared__ ST r_sc[32];
  __shared__ int32_t r_c[32];
  __shared__ int64_t r_kid[32];
  __shared__ int32_t s_mv;
  __shared__ unsigned s_nused[2];
  typedef typename TableVal<ST>::type VT;
  const int Hmax = 1 << log2H;
  VT *vals = reinterpret_cast<VT *>(smem);
  int32_t *keys = reinterpret_cast<int32_t *>(vals + Hmax);
  uint16_t *used = reinterpret_cast<uint16_t *>(keys + Hmax);   // Hmax / 2 entries
  // the warps' combine scratch follows, 32 words per warp of this block (sized
  // by the launch, so small blocks keep their shared memory small)
  u64 (*wscratch)[32] = reinterpret_cast<u64 (*)[32]>(used + Hmax / 2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int64_t scanned = 0, nvert = 0, ncand = 0, nmoves = 0;
  i128 accS = 0;
  for (int s = threadIdx.x; s < Hmax; s += blockDim.x) { keys[s] = LEIDEN_EMPTY_KEY; vals[s] = 0; }
  if (threadIdx.x < 2) s_nused[threadIdx.x] = 0;
  int par = 0;   // parity of the vertices this block has decided
  int bpar = 0;  // parity of the staged batches
  const int64_t stride = gridDim.x;
  for (int64_t base = blockIdx.x; base < a.list_n; base += 32 * stride, bpar ^= 1) {
    if (warp == 0) {
      // header loads as in the group tiers, one listed vertex per lane
      const int64_t li = base + (int64_t)lane * stride;
      const bool valid = li < a.list_n;
      const int32_t i = valid ? a.list[li] : 0;
      int64_t h0 = 0, h1 = 0, hK = 0, hSd = 0;
      int32_t hd = 0;
      if (a.spec && valid) {
        h0 = a.g.off[i];
        h1 = a.g.off[i + 1];
        hd = a.C[i];
        hK = a.K[i];
        if (!ASYNC) hSd = a.Sig[hd];
      }
      const bool act = valid && eligible<REFINE>(a, i);
      if (!a.spec && act) {
        h0 = a.g.off[i];
        h1 = a.g.off[i + 1];
        hd = a.C[i];
        hK = a.K[i];
        if (!ASYNC) hSd = a.Sig[hd];
      }
      const unsigned m = __ballot_sync(FULL_MASK, act);
      if (act) {
        const int pos = __popc(m & ((1u << lane) - 1u));
        h_i[pos] = i;
        h_d[pos] = hd;
        h_e0[pos] = h0;
        h_e1[pos] = h1;
        h_K[pos] = hK;
        h_Sd[pos] = hSd;
      }
      if (lane == 0) s_nact[bpar] = __popc(m);
    }
    __syncthreads();
    const int nact = s_nact[bpar];
    for (int k = 0; k < nact; k++, par ^= 1) {
      const int32_t i = h_i[k], d = h_d[k];
      const int64_t e0 = h_e0[k], e1 = h_e1[k];
      // table sized for this row: at least 2 * degree slots, at most the tier's
      int lh = 1;
      while (lh < log2H && ((int64_t)1 << lh) < 2 * (e1 - e0)) lh++;
      const int32_t cbi = REFINE ? a.CB[i] : 0;
      // each warp walks 32-entry chunks (warp-uniform), combining equal
      // communities across its lanes before the atomics
      for (int64_t cb = e0 + 32 * warp; cb < e1; cb += 32 * (int64_t)nwarp * BLOCK_ROW_UNROLL) {
        int32_t cc[BLOCK_ROW_UNROLL];
        u64 wv[BLOCK_ROW_UNROLL];
#pragma unroll
        for (int u = 0; u < BLOCK_ROW_UNROLL; u++) {
          const int64_t e = cb + (int64_t)u * 32 * nwarp + lane;
          const bool in = e < e1;
          const int32_t j = in ? a.g.idx[e] : -1;
          wv[u] = in ? (u64)(int64_t)a.g.w[e] : 0;
          bool ok = in && j != i;
          if (ok && (uint32_t)j >= (uint32_t)a.g.n) { atomicOr(&a.ctr[CTR_ERROR], 64ull); ok = false; }
          cc[u] = ok ? j : -1;
        }
#pragma unroll
        for (int u = 0; u < BLOCK_ROW_UNROLL; u++) {
          const int32_t j = cc[u];
          bool ok = j >= 0;
          if (REFINE && ok && a.CB[j] != cbi) ok = false;
          cc[u] = ok ? a.C[j] : LEIDEN_EMPTY_KEY;
        }
#pragma unroll
        for (int u = 0; u < BLOCK_ROW_UNROLL; u++) {
          u64 sum = 0;
          int slot = -1;
          if (warp_combine((unsigned long long)(uint32_t)cc[u], cc[u] != LEIDEN_EMPTY_KEY, wv[u], &sum,
                           wscratch[warp]))
            slot = table_add_new(keys, vals, lh, cc[u], sum, &a.ctr[CTR_ERROR]);
          list_new_slots(slot, used, &s_nused[par]);
        }
      }
      if (threadIdx.x == 0) { scanned += e1 - e0; nvert++; }
      __syncthreads();
      const unsigned nused = s_nused[par];
      const ST A = (ST)a.A;
      const int64_t Ki = h_K[k];
      const ST B = (ST)a.p * (ST)Ki;
      ST bsc = 0;
      int32_t bc = INT32_MAX;
      int64_t kid = 0;
      for (unsigned u = threadIdx.x; u < nused; u += blockDim.x) {
        const uint32_t sl = used[u];
        const int32_t c = keys[sl];
        const int64_t v = (int64_t)vals[sl];
        keys[sl] = LEIDEN_EMPTY_KEY;   // reset on read: clean for the next vertex
        vals[sl] = 0;
        ncand++;
        if (c == d) { kid = v; continue; }
        const ST sc = A * (ST)v - B * (ST)sigma_for_score(a.Sig, c);
        if (better(sc, c, bsc, bc)) { bsc = sc; bc = c; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const ST osc = shfl_xor_any<ST>(bsc, o);
        const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
        kid += shfl_xor_i64(kid, o);
        if (better(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
      }
      if (lane == 0) { r_sc[warp] = bsc; r_c[warp] = bc; r_kid[warp] = kid; }
      const int64_t Sd = h_Sd[k];
      __syncthreads();
      if (warp == 0) {
        // the warps' bests, combined by warp 0 alone: the others go on to the
        // next row (r_* are rewritten only after the next row's barrier)
        bsc = lane < nwarp ? r_sc[lane] : (ST)0;
        bc = lane < nwarp ? r_c[lane] : INT32_MAX;
        kid = lane < nwarp ? r_kid[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const ST osc = shfl_xor_any<ST>(bsc, o);
          const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
          kid += shfl_xor_i64(kid, o);
          if (better(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
        }
        if (lane == 0) {
          s_nused[par] = 0;   // for the row after next
          bool propose = false;
          i128 S = 0;
          if (bc != INT32_MAX) {
            S = (i128)bsc - (i128)a.A * kid - (i128)a.p * Ki * (Ki - (ASYNC ? a.Sig[d] : Sd));
            propose = S > 0;
            if (REFINE && propose && a.C[bc] != bc) propose = false;
          }
          if (ASYNC) {
            if (propose) propose = commit_async<REFINE>(a, i, d, bc);
            if (propose) { accS += S; nmoves++; }
          } else if (propose) {
            const u64 slot = atomicAdd(a.prop_count, 1ull);
            a.prop_i[slot] = i;
            a.prop_c[slot] = bc;
            a.prop_S[slot] = S;
            if (REFINE) a.stamp[i] = a.stamp_val;
          }
          s_mv = propose;
        }
      }
      if (ASYNC && !REFINE) {
        __syncthreads();
        if (s_mv)
          for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) unmark(a.processed, a.g.idx[e]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    scanned += shfl_xor_i64(scanned, o);
    nvert += shfl_xor_i64(nvert, o);
    ncand += shfl_xor_i64(ncand, o);
  }
  if (lane == 0) {
    if (scanned) atomicAdd(&a.ctr[CTR_SCANNED_ENTRIES], (u64)scanned);
    if (nvert) atomicAdd(&a.ctr[CTR_SCANNED_VERTICES], (u64)nvert);
    if (ncand) atomicAdd(&a.ctr[CTR_CANDIDATES], (u64)ncand);
  }
  if (ASYNC && threadIdx.x == 0 && nmoves) {
    atomicAdd(&a.ctr[CTR_MOVES], (u64)nmoves);
    atomic_add_i128(&a.ctr[CTR_SUMS_LO], accS);
  }
}

// ---------------------------------------------------------------------------
// DET apply kernels.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) apply_moves_k(const int32_t *prop_i, const int32_t *prop_c,
                                                     const i128 *prop_S, u64 *ctr, int32_t *C,
                                                     const int64_t *K, int64_t *Sig, uint8_t *changed,
                                                     uint8_t *processed, const int64_t *off,
                                                     const int32_t *idx, int32_t *big, int dynamic) {
  __shared__ i128 sbuf[32];
  const u64 cnt = ctr[CTR_PROPS];
  const int lane = threadIdx.x & 31;
  const u64 gt = (u64)blockIdx.x * blockDim.x + threadIdx.x, nt = (u64)gridDim.x * blockDim.x;
  i128 acc = 0;
  // commits: one thread per proposal (the vertex's own entries only)
  for (u64 m = gt; m < cnt; m += nt) {
    const int32_t i = prop_i[m], c = prop_c[m];
    const int32_t d = C[i];
    const int64_t Ki = K[i];
    atomic_add_i64(&Sig[d], -Ki);
    atomic_add_i64(&Sig[c], Ki);
    C[i] = c;
    if (dynamic) { changed[d] = 1; changed[c] = 1; }
    acc += prop_S[m];
  }
  // vertex pruning: a mover re-marks its neighbours, half a warp per mover
  // with four row loads in flight (independent of the commits above; long
  // rows are left to the big-row kernel, which spreads them over the grid)
  const u64 hw_glob = gt >> 4, nhw = nt >> 4;
  const int hl = lane & 15;
  for (u64 m = hw_glob; m < cnt; m += nhw) {
    const int32_t i = prop_i[m];
    const int64_t e0 = off[i];
    int64_t e1 = off[i + 1];
    if (e1 - e0 > BIG_ROW) {
      if (hl == 0) big[atomicAdd(&ctr[CTR_BIG], 1ull)] = i;
      e1 = e0;
    }
    constexpr int RU = LK_REMARK_UNROLL;
    for (int64_t e = e0 + hl; e < e1; e += 16 * RU) {
      int32_t j[RU];
#pragma unroll
      for (int u = 0; u < RU; u++) j[u] = e + 16 * u < e1 ? idx[e + 16 * u] : -1;
      // most neighbours of a mover are re-marked already (by an earlier
      // mover of the sub-sweep): reading the flag first spares the store,
      // and the random byte stores were what held the kernel back (Chung-Lu
      // Static 2382 -> 2185 ms)
      uint8_t f[RU];
#pragma unroll
      for (int u = 0; u < RU; u++) f[u] = j[u] >= 0 ? processed[j[u]] : 0;
#pragma unroll
      for (int u = 0; u < RU; u++)
        if (f[u]) processed[j[u]] = 0;
    }
  }
  const i128 tot = block_sum_i128(acc, sbuf);
  if (threadIdx.x == 0 && tot != 0) atomic_add_i128(&ctr[CTR_SUMS_LO], tot);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctr[CTR_MOVES], cnt);
}

__global__ void __launch_bounds__(256) apply_refine_k(const int32_t *prop_i, const int32_t *prop_c,
                                                      u64 *ctr, const uint8_t *stamp, uint8_t sv,
                                                      int32_t *C, const int64_t *K, int64_t *Sig) {
  const u64 cnt = ctr[CTR_PROPS];
  u64 moved = 0;
  for (u64 m = (u64)blockIdx.x * blockDim.x + threadIdx.x; m < cnt; m += (u64)gridDim.x * blockDim.x) {
    const int32_t i = prop_i[m], c = prop_c[m];
    if (stamp[c] == sv) continue;   // the target proposed to leave in this sub-sweep
    const int64_t Ki = K[i];
    atomic_add_i64(&Sig[i], -Ki);   // C'[i] = i: Sigma'[i] drops to 0
    atomic_add_i64(&Sig[c], Ki);
    C[i] = c;
    moved++;
  }
  for (int o = 16; o > 0; o >>= 1) moved += __shfl_xor_sync(FULL_MASK, moved, o);
  if ((threadIdx.x & 31) == 0 && moved) atomicAdd(&ctr[CTR_MOVES], moved);
}

void launch_apply_moves(const int32_t *prop_i, const int32_t *prop_c, const i128 *prop_S,
                        u64 *ctr, int32_t *C, const int64_t *K, int64_t *Sig,
                        uint8_t *changed, uint8_t *processed, const int64_t *off,
                        const int32_t *idx, int32_t *big, int dynamic, int sms, cudaStream_t s) {
  const unsigned grid = (unsigned)resident_blocks((const void *)apply_moves_k, 256, 0, sms);
  LK_COUNTED apply_moves_k<<<grid, 256, 0, s>>>(prop_i, prop_c, prop_S, ctr, C, K, Sig, changed,
                                        processed, off, idx, big, dynamic);
}

void launch_apply_refine(const int32_t *prop_i, const int32_t *prop_c, u64 *ctr,
                         const uint8_t *stamp, uint8_t sv, int32_t *C, const int64_t *K,
                         int64_t *Sig, int sms, cudaStream_t s) {
  LK_COUNTED apply_refine_k<<<sms * 2, 256, 0, s>>>(prop_i, prop_c, ctr, stamp, sv, C, K, Sig);
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <int G, int LOG2H, bool REFINE, bool ASYNC, typename WT, typename ST>
static void launch_group_k(const Tier &t, const MoveArgs<WT> &a, int sms, cudaStream_t s) {
  auto k = decide_group<G, LOG2H, REFINE, ASYNC, WT, ST>;
  const int threads = t.threads;
  const size_t smem = (size_t)(threads / 32) * (32 / G) * (1u << LOG2H) *
                      (sizeof(typename TableVal<ST>::type) + sizeof(int32_t));
  ensure_smem((const void *)k, smem);
  const int64_t groups_per_block = (threads / 32) * (32 / G);
  int64_t blocks = (a.list_n + groups_per_block - 1) / groups_per_block;
  const int64_t cap = resident_blocks((const void *)k, threads, smem, sms);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  LK_COUNTED k<<<(unsigned)blocks, threads, smem, s>>>(a);
}

template <typename WT, typename ST, bool REFINE, bool ASYNC>
void launch_decide(const Tier &t, const MoveArgs<WT> &a, int sms, cudaStream_t s) {
  if (a.list_n <= 0) return;
  // A whole-warp group tier with rows of more than 64 entries and too few
  // vertices to fill the GPU runs in a single wave, so its time is one
  // vertex's latency: give each vertex a block of four warps instead (same
  // decisions, a quarter of the per-vertex steps).
  if (t.kind == TIER_GROUP && t.G == 32 && t.log2H >= 8 && a.list_n <= (int64_t)sms * SMALL_WAVE_VERTICES) {
    const Tier b{TIER_BLOCK, t.maxdeg, 0, t.log2H, 128};
    launch_decide<WT, ST, REFINE, ASYNC>(b, a, sms, s);
    return;
  }
  if (t.kind == TIER_GROUP && t.G == 1) {
    // one lane per vertex; log2H holds the register capacity, 4 or 8 entries
    int64_t blocks = (a.list_n + t.threads - 1) / t.threads;
    const int64_t cap = (int64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (t.log2H == 2) LK_COUNTED decide_thread<4, REFINE, ASYNC, WT, ST><<<(unsigned)blocks, t.threads, 0, s>>>(a);
    else if (t.log2H == 3) LK_COUNTED decide_thread<8, REFINE, ASYNC, WT, ST><<<(unsigned)blocks, t.threads, 0, s>>>(a);
    return;
  }
  if (t.kind == TIER_GROUP) {
#define LK_GROUP(GG, LH)                                                        \
  if (t.G == GG && t.log2H == LH) {                                             \
    launch_group_k<GG, LH, REFINE, ASYNC, WT, ST>(t, a, sms, s);                \
    return;                                                                     \
  }
    LK_GROUP(4, 3) LK_GROUP(4, 4) LK_GROUP(8, 4) LK_GROUP(8, 5) LK_GROUP(16, 5) LK_GROUP(16, 6)
    LK_GROUP(32, 6) LK_GROUP(32, 7) LK_GROUP(32, 8) LK_GROUP(32, 9) LK_GROUP(32, 10)
#undef LK_GROUP
    return;  // unsupported combination: the tier table is validated on the host
  }
  if (t.kind != TIER_BLOCK) return;  // hub rows go through launch_hubs
  const int log2H = t.log2H;
  // table (value, key), the list of used slots (at most half the table) and
  // the warps' combine scratch
  const size_t smem = (size_t)(1u << log2H) * (sizeof(typename TableVal<ST>::type) + sizeof(int32_t)) +
                      (size_t)(1u << log2H) + (size_t)(t.threads / 32) * 32 * sizeof(u64);
  auto k = decide_block<REFINE, ASYNC, WT, ST>;
  ensure_smem((const void *)k, smem);
  // one listed vertex per block at a time: as many blocks as fit on the SMs
  // at once (more would run as a partial second wave of grid-stride shares)
  int64_t blocks = a.list_n;
  const int64_t cap = resident_blocks((const void *)k, t.threads, smem, sms);
  if (blocks > cap) blocks = cap;
  LK_COUNTED k<<<(unsigned)blocks, t.threads, smem, s>>>(a, log2H);
}

#define LK_INST(WT, ST)                                                                          \
  template void launch_decide<WT, ST, false, false>(const Tier &, const MoveArgs<WT> &, int, cudaStream_t); \
  template void launch_decide<WT, ST, true, false>(const Tier &, const MoveArgs<WT> &, int, cudaStream_t);  \
  template void launch_decide<WT, ST, false, true>(const Tier &, const MoveArgs<WT> &, int, cudaStream_t);  \
  template void launch_decide<WT, ST, true, true>(const Tier &, const MoveArgs<WT> &, int, cudaStream_t);
LK_INST(int32_t, int64_t)
LK_INST(int32_t, i128)
LK_INST(int64_t, int64_t)
LK_INST(int64_t, i128)
#undef LK_INST

TierTable default_tiers() {
  TierTable tt{};
  int k = 0;
  tt.t[k++] = {TIER_SKIP, 0, 0, 0, 0};
  // rows of up to 8 entries: one lane per vertex, the row in registers
  tt.t[k++] = {TIER_GROUP, 4, 1, 2, 256};
  tt.t[k++] = {TIER_GROUP, 8, 1, 3, 256};
  tt.t[k++] = {TIER_GROUP, 16, 16, 5, 256};
  tt.t[k++] = {TIER_GROUP, 32, 32, 6, 256};
  tt.t[k++] = {TIER_GROUP, 128, 32, 8, 256};
  tt.t[k++] = {TIER_GROUP, 256, 32, 9, 256};
  // rows of 257..512 entries on 4-warp blocks: measured 152 against 156 ms
  // for one warp each (R-MAT scale 22 Static)
  tt.t[k++] = {TIER_BLOCK, 512, 0, 10, 128};
  tt.t[k++] = {TIER_BLOCK, 2048, 0, 12, 256};
  tt.t[k++] = {TIER_BLOCK, 8192, 0, 14, 512};
  tt.t[k++] = {TIER_GLOBAL, INT64_MAX, 0, 0, 1024};
  tt.ntiers = k;
  return tt;
}

}  // namespace lk
