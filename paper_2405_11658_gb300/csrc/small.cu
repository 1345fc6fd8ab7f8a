// small.cu -- many small graphs in one persistent launch (leiden_batch_run).
//
// Each thread block runs the whole of Alg. leiden for one graph at a time --
// marking (Alg. frontier / naive), every pass of local-moving (Alg. leidenlm,
// DET sub-sweeps), subset renumbering (Alg. leidensr), the break of changed
// communities, refinement (Alg. leidenre), renumbering, aggregation
// (Alg. leidenag), the dendrogram lookup, canonical labels and the terms of
// Eq. 1 -- then takes the next graph from a device-side queue.  Phases are
// separated by __syncthreads only; nothing waits on another block.
//
// The arithmetic and the schedule are those of the multi-kernel path: the
// integer score of Eq. 2 scaled by 2m^2 (128-bit here for every graph), ties
// to the smallest community ID, colour classes by the top bits of
// (uint32)(i * 2654435761), moves of a class decided against the state at
// its start and applied together, refinement proposals accepted only when
// the target made none.  So each graph ends with the same membership and
// statistics as leiden_static / leiden_update give it.
//
// Rows of up to SB_WARP_SLOTS / 2 entries are hashed by one warp into a
// shared-memory table; longer rows (and communities of the aggregation) by
// the whole block into the graph's table in global scratch.
#include <limits.h>

#include "common.cuh"
#include "internal.h"
#include "small.h"

namespace lk {

namespace {

constexpr int SB_WARP_SLOTS = 256;   // shared-memory slots per warp
constexpr int SB_GROUP_ROW = 32;     // rows up to this long go to 8-lane groups (64-slot tables)
constexpr int SB_MAX_WARPS = 32;
constexpr int SB_MAX_CLASSES = 256;

// ---------------------------------------------------------------------------
// Correctly rounded int128 -> double (round to nearest even) by round-to-odd
// double rounding (Boldo and Melquiond, "When double rounding is odd", 2005):
// truncate to the top 64 significant bits and OR every dropped bit into the
// lowest kept bit (the sticky bit), which rounds the value to odd at 64 bits;
// then convert those 64 bits to double (round to nearest even) and scale by
// the dropped power of two.  A round-to-odd intermediate with at least two
// more bits than the 53-bit target makes the second rounding equal to a
// single correct rounding of the original value.
// ---------------------------------------------------------------------------
__device__ double i128_to_double(i128 x) {
  const bool neg = x < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-(x + 1)) + 1u : (unsigned __int128)x;
  const u64 hi = (u64)(u >> 64);
  double r;
  if (hi == 0) {
    r = __ull2double_rn((u64)u);
  } else {
    const int s = 64 - __clzll((long long)hi);   // bits beyond the low 64
    const u64 top = (u64)(u >> s);
    const bool sticky = (u & (((unsigned __int128)1 << s) - 1u)) != 0;
    r = ldexp(__ull2double_rn(top | (sticky ? 1ull : 0ull)), s);
  }
  return neg ? -r : r;
}

template <typename WT>
struct Lvl {
  int64_t n;
  const int64_t *off;
  const int32_t *idx;
  const WT *w;
};

struct Shared {
  int job;
  int stop;
  u64 err;
  unsigned nprop, nlong, nmed;
  int64_t long_n;
  int32_t koff[SB_MAX_CLASSES + 1];
  int32_t kcur[SB_MAX_CLASSES];
  i128 red128[SB_MAX_WARPS];
  int64_t red64[SB_MAX_WARPS];
  int32_t redc[SB_MAX_WARPS];
  u64 wscr[SB_MAX_WARPS][32];
};

// Per-run constants of one graph.
struct Ctl {
  int64_t A;       // 2m * q
  int64_t p, q, two_m;
  double den;      // (2m)^2 / 2 * q
  int log2S;
  int dynamic;     // changed flags follow the moves (first pass of ND / DS / DF)
  const uint8_t *in_range;  // DS affected range in the first pass, else NULL
};

__device__ __forceinline__ bool better128(i128 sc, int32_t c, i128 bsc, int32_t bc) {
  return c != INT32_MAX && (bc == INT32_MAX || sc > bsc || (sc == bsc && c < bc));
}

__device__ __forceinline__ void tbl_add(int32_t *keys, u64 *vals, int64_t log2H, int32_t c, u64 w, u64 *err) {
  const uint64_t mask = ((uint64_t)1 << log2H) - 1u;
  uint64_t s = (uint64_t)(hash32(c) >> (32 - log2H));
  for (uint64_t probe = 0; probe <= mask; probe++) {
    const int32_t k = *(volatile int32_t *)&keys[s];
    if (k == c) { atomicAdd(&vals[s], w); return; }
    if (k == LEIDEN_EMPTY_KEY) {
      const int32_t old = atomicCAS(&keys[s], LEIDEN_EMPTY_KEY, c);
      if (old == LEIDEN_EMPTY_KEY || old == c) { atomicAdd(&vals[s], w); return; }
    }
    s = (s + 1) & mask;
  }
  atomicOr(err, 16ull);
}

__device__ __forceinline__ int log2_at_least(int64_t x) {  // smallest k >= 1 with 2^k >= x
  int k = 1;
  while (((int64_t)1 << k) < x) k++;
  return k;
}

// Block-wide sums; every thread calls, every thread gets the result.
__device__ i128 bsum128(i128 v, Shared &sm) {
  for (int o = 16; o; o >>= 1) v += shfl_xor_i128(v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm.red128[warp] = v;
  __syncthreads();
  i128 r = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) r += sm.red128[k];
  __syncthreads();
  return r;
}
__device__ int64_t bsum64(int64_t v, Shared &sm) {
  for (int o = 16; o; o >>= 1) v += shfl_xor_i64(v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sm.red64[warp] = v;
  __syncthreads();
  int64_t r = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) r += sm.red64[k];
  __syncthreads();
  return r;
}

// Block-wide exclusive scan of in[0..n) (any integer type) into out[0..n],
// out[n] = total.  Tiles of blockDim.x elements with a running carry.
template <typename T>
__device__ void bscan(const T *in, int64_t *out, int64_t n, Shared &sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t k = base + threadIdx.x;
    const int64_t v = k < n ? (int64_t)in[k] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = shfl_i64(x, (lane - o) & 31);
      if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sm.red64[warp] = x;
    __syncthreads();
    int64_t pre = carry;
    for (int q = 0; q < warp; q++) pre += sm.red64[q];
    if (k < n) out[k] = pre + x - v;
    int64_t tile = 0;
    for (int q = 0; q < nw; q++) tile += sm.red64[q];
    carry += tile;
  }
  __syncthreads();
  if (threadIdx.x == 0) out[n] = carry;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Workspace of one graph, carved from its slice of the batch arena.
// ---------------------------------------------------------------------------
struct WS {
  int32_t *Ctop, *Cp, *CB, *rep, *vl, *pi, *pc, *cv, *longl, *gkeys, *idxA, *idxB, *hidx;
  int64_t *Kp, *Sp, *S2, *scn, *coff, *ccur, *hoff, *cdist, *offA, *offB, *wA, *wB, *hw;
  i128 *pS;
  uint8_t *ch, *ch2, *proc, *stamp, *flag;
  u64 *gvals;
  int log2T;
};

__device__ void carve_ws(char *base, int64_t n, int64_t nnz, WS &w) {
  SmallLayout L = small_layout(n, nnz);
  w.Ctop = (int32_t *)(base + L.Ctop); w.Cp = (int32_t *)(base + L.Cp); w.CB = (int32_t *)(base + L.CB);
  w.rep = (int32_t *)(base + L.rep); w.vl = (int32_t *)(base + L.vl); w.pi = (int32_t *)(base + L.pi);
  w.pc = (int32_t *)(base + L.pc); w.cv = (int32_t *)(base + L.cv); w.longl = (int32_t *)(base + L.longl);
  w.gkeys = (int32_t *)(base + L.gkeys); w.idxA = (int32_t *)(base + L.idxA); w.idxB = (int32_t *)(base + L.idxB);
  w.hidx = (int32_t *)(base + L.hidx);
  w.Kp = (int64_t *)(base + L.Kp); w.Sp = (int64_t *)(base + L.Sp); w.S2 = (int64_t *)(base + L.S2);
  w.scn = (int64_t *)(base + L.scn); w.coff = (int64_t *)(base + L.coff); w.ccur = (int64_t *)(base + L.ccur);
  w.hoff = (int64_t *)(base + L.hoff); w.cdist = (int64_t *)(base + L.cdist); w.offA = (int64_t *)(base + L.offA);
  w.offB = (int64_t *)(base + L.offB); w.wA = (int64_t *)(base + L.wA); w.wB = (int64_t *)(base + L.wB);
  w.hw = (int64_t *)(base + L.hw);
  w.pS = (i128 *)(base + L.pS);
  w.ch = (uint8_t *)(base + L.ch); w.ch2 = (uint8_t *)(base + L.ch2); w.proc = (uint8_t *)(base + L.proc);
  w.stamp = (uint8_t *)(base + L.stamp); w.flag = (uint8_t *)(base + L.flag);
  w.gvals = (u64 *)(base + L.gvals);
  w.log2T = L.log2T;
}

// ---------------------------------------------------------------------------
// Decisions of colour class [kb, ke) of the vertex list: local-moving
// (REFINE = false) or refinement (REFINE = true).  Proposals go to
// (pi, pc, pS)[0 .. sm.nprop).
// ---------------------------------------------------------------------------
// Proposal of vertex i (one thread): Eq. 2 scaled, the move rule and, for
// refinement, the target's own vertex still in place.
template <bool REFINE>
__device__ __forceinline__ void propose_move(WS &w, const Ctl &ct, int32_t i, int32_t d, i128 bsc, int32_t bc,
                                             int64_t kid, uint8_t sv, Shared &sm) {
  if (bc == INT32_MAX) return;
  const int64_t Ki = w.Kp[i];
  const i128 S = bsc - (i128)ct.A * kid - (i128)ct.p * Ki * (Ki - w.Sp[d]);
  bool propose = S > 0;
  if (REFINE && propose && w.Cp[bc] != bc) propose = false;
  if (!propose) return;
  const unsigned slot = atomicAdd(&sm.nprop, 1u);
  w.pi[slot] = i;
  w.pc[slot] = bc;
  w.pS[slot] = S;
  if (REFINE) w.stamp[i] = sv;
}

template <bool REFINE, typename WT>
__device__ void decide(const Lvl<WT> &g, WS &w, const Ctl &ct, int32_t kb, int32_t ke, uint8_t sv,
                       int32_t *skeys_all, u64 *svals_all, Shared &sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) { sm.nprop = 0; sm.nlong = 0; sm.nmed = 0; }
  __syncthreads();
  // Rows of at most SB_GROUP_ROW entries: groups of 8 lanes, four vertices per
  // warp, a 64-slot table each.  Longer rows are set aside: up to half the
  // warp table for the warp pass below, the rest for the block pass.
  {
    constexpr int G = 8, GPW = 32 / G, GS = SB_WARP_SLOTS / GPW;
    const int gw = lane / G, gl = lane % G, leader = gw * G;
    int32_t *gkeys = skeys_all + warp * SB_WARP_SLOTS + gw * GS;
    u64 *gvals = svals_all + warp * SB_WARP_SLOTS + gw * GS;
    for (int32_t kb2 = kb + warp * GPW; kb2 < ke; kb2 += nw * GPW) {  // uniform per warp
      const int32_t k = kb2 + gw;
      const bool valid = k < ke;
      const int32_t i = valid ? w.vl[k] : 0;
      bool act = false;
      if (gl == 0 && valid) {
        if (!REFINE) {
          act = !w.proc[i];
          w.proc[i] = 1;
          if (act && ct.in_range) act = ct.in_range[i] != 0;   // inAffectedRange (Alg. delta)
        } else {
          act = w.ch[w.CB[i]] && w.Cp[i] == i && w.Sp[i] == w.Kp[i];
        }
      }
      act = __shfl_sync(FULL_MASK, act, leader);
      int64_t e0 = 0, e1 = 0;
      if (act) { e0 = g.off[i]; e1 = g.off[i + 1]; }
      if (act && e1 - e0 > SB_GROUP_ROW) {
        if (gl == 0) {
          if (2 * (e1 - e0) > SB_WARP_SLOTS) w.longl[atomicAdd(&sm.nlong, 1u)] = i;
          else w.cv[atomicAdd(&sm.nmed, 1u)] = i;
        }
        act = false;
      }
      int lh = 1;
      if (act) {
        lh = log2_at_least(2 * (e1 - e0));
        for (int s2 = gl; s2 < (1 << lh); s2 += G) { gkeys[s2] = LEIDEN_EMPTY_KEY; gvals[s2] = 0; }
      }
      __syncwarp();
      const int32_t d = act ? w.Cp[i] : 0;
      const int32_t cbi = (REFINE && act) ? w.CB[i] : 0;
      int64_t span = act ? e1 - e0 : 0;
      for (int o = 16; o; o >>= 1) {
        const int64_t y = shfl_xor_i64(span, o);
        span = y > span ? y : span;
      }
      for (int64_t xb = 0; xb < span; xb += G) {  // uniform per warp
        const int64_t e = e0 + xb + gl;
        const bool in = act && e < e1;
        const int32_t j = in ? g.idx[e] : -1;
        const u64 wv = in ? (u64)(int64_t)g.w[e] : 0;
        bool ok = in && j != i;
        if (REFINE && ok && w.CB[j] != cbi) ok = false;
        const int32_t c = ok ? w.Cp[j] : LEIDEN_EMPTY_KEY;
        u64 sum = 0;
        const unsigned long long key = ((unsigned long long)(uint32_t)gw << 32) | (uint32_t)c;
        if (warp_combine(key, ok, wv, &sum, sm.wscr[warp])) tbl_add(gkeys, gvals, lh, c, sum, &sm.err);
      }
      __syncwarp();
      i128 bsc = 0;
      int32_t bc = INT32_MAX;
      int64_t kid = 0;
      if (act) {
        const i128 A = (i128)ct.A;
        const i128 B = (i128)ct.p * (i128)w.Kp[i];
        for (int s2 = gl; s2 < (1 << lh); s2 += G) {
          const int32_t c = gkeys[s2];
          if (c == LEIDEN_EMPTY_KEY) continue;
          const int64_t v = (int64_t)gvals[s2];
          if (c == d) { kid = v; continue; }
          const i128 sc = A * (i128)v - B * (i128)w.Sp[c];
          if (better128(sc, c, bsc, bc)) { bsc = sc; bc = c; }
        }
      }
      for (int o = G / 2; o; o >>= 1) {
        const i128 osc = shfl_xor_i128(bsc, o);
        const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
        kid += shfl_xor_i64(kid, o);
        if (better128(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
      }
      if (act && gl == 0) propose_move<REFINE>(w, ct, i, d, bsc, bc, kid, sv, sm);
      __syncwarp();
    }
  }
  __syncthreads();
  // medium rows: one warp each, a table of up to SB_WARP_SLOTS slots
  int32_t *keys = skeys_all + warp * SB_WARP_SLOTS;
  u64 *vals = svals_all + warp * SB_WARP_SLOTS;
  const unsigned nmed = sm.nmed;
  for (unsigned t = warp; t < nmed; t += nw) {
    const int32_t i = w.cv[t];
    const int64_t e0 = g.off[i], e1 = g.off[i + 1];
    const int lh = log2_at_least(2 * (e1 - e0));
    for (int s = lane; s < (1 << lh); s += 32) { keys[s] = LEIDEN_EMPTY_KEY; vals[s] = 0; }
    __syncwarp();
    const int32_t d = w.Cp[i];
    const int32_t cbi = REFINE ? w.CB[i] : 0;
    for (int64_t xb = 0; xb < e1 - e0; xb += 32) {
      const int64_t e = e0 + xb + lane;
      const bool in = e < e1;
      const int32_t j = in ? g.idx[e] : -1;
      const u64 wv = in ? (u64)(int64_t)g.w[e] : 0;
      bool ok = in && j != i;
      if (REFINE && ok && w.CB[j] != cbi) ok = false;
      const int32_t c = ok ? w.Cp[j] : LEIDEN_EMPTY_KEY;
      u64 sum = 0;
      if (warp_combine((unsigned long long)(uint32_t)c, ok, wv, &sum, sm.wscr[warp]))
        tbl_add(keys, vals, lh, c, sum, &sm.err);
    }
    __syncwarp();
    const i128 A = (i128)ct.A;
    const i128 B = (i128)ct.p * (i128)w.Kp[i];
    i128 bsc = 0;
    int32_t bc = INT32_MAX;
    int64_t kid = 0;
    for (int s = lane; s < (1 << lh); s += 32) {
      const int32_t c = keys[s];
      if (c == LEIDEN_EMPTY_KEY) continue;
      const int64_t v = (int64_t)vals[s];
      if (c == d) { kid = v; continue; }
      const i128 sc = A * (i128)v - B * (i128)w.Sp[c];
      if (better128(sc, c, bsc, bc)) { bsc = sc; bc = c; }
    }
    for (int o = 16; o; o >>= 1) {
      const i128 osc = shfl_xor_i128(bsc, o);
      const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
      kid += shfl_xor_i64(kid, o);
      if (better128(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
    }
    if (lane == 0) propose_move<REFINE>(w, ct, i, d, bsc, bc, kid, sv, sm);
    __syncwarp();
  }
  __syncthreads();
  // long rows: the whole block per row, table in global scratch
  const unsigned nlong = sm.nlong;
  for (unsigned t = 0; t < nlong; t++) {
    const int32_t i = w.longl[t];
    const int64_t e0 = g.off[i], e1 = g.off[i + 1];
    const int64_t cap = (e1 - e0) < g.n ? (e1 - e0) : g.n;
    int lh = log2_at_least(2 * cap);
    if (lh > w.log2T) { if (threadIdx.x == 0) atomicOr(&sm.err, 32ull); lh = w.log2T; }
    for (int64_t s = threadIdx.x; s < ((int64_t)1 << lh); s += blockDim.x) {
      w.gkeys[s] = LEIDEN_EMPTY_KEY;
      w.gvals[s] = 0;
    }
    __syncthreads();
    const int32_t d = w.Cp[i];
    const int32_t cbi = REFINE ? w.CB[i] : 0;
    for (int64_t cb = e0 + 32 * warp; cb < e1; cb += 32 * (int64_t)nw) {
      const int64_t e = cb + lane;
      const bool in = e < e1;
      const int32_t j = in ? g.idx[e] : -1;
      const u64 wv = in ? (u64)(int64_t)g.w[e] : 0;
      bool ok = in && j != i;
      if (REFINE && ok && w.CB[j] != cbi) ok = false;
      const int32_t c = ok ? w.Cp[j] : LEIDEN_EMPTY_KEY;
      u64 sum = 0;
      if (warp_combine((unsigned long long)(uint32_t)c, ok, wv, &sum, sm.wscr[warp]))
        tbl_add(w.gkeys, w.gvals, lh, c, sum, &sm.err);
    }
    __syncthreads();
    const i128 A = (i128)ct.A;
    const i128 B = (i128)ct.p * (i128)w.Kp[i];
    i128 bsc = 0;
    int32_t bc = INT32_MAX;
    int64_t kid = 0;
    for (int64_t s = threadIdx.x; s < ((int64_t)1 << lh); s += blockDim.x) {
      const int32_t c = w.gkeys[s];
      if (c == LEIDEN_EMPTY_KEY) continue;
      const int64_t v = (int64_t)w.gvals[s];
      if (c == d) { kid = v; continue; }
      const i128 sc = A * (i128)v - B * (i128)w.Sp[c];
      if (better128(sc, c, bsc, bc)) { bsc = sc; bc = c; }
    }
    for (int o = 16; o; o >>= 1) {
      const i128 osc = shfl_xor_i128(bsc, o);
      const int32_t oc = __shfl_xor_sync(FULL_MASK, bc, o);
      kid += shfl_xor_i64(kid, o);
      if (better128(osc, oc, bsc, bc)) { bsc = osc; bc = oc; }
    }
    if (lane == 0) { sm.red128[warp] = bsc; sm.redc[warp] = bc; sm.red64[warp] = kid; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < nw; q++) {
        kid += sm.red64[q];
        if (better128(sm.red128[q], sm.redc[q], bsc, bc)) { bsc = sm.red128[q]; bc = sm.redc[q]; }
      }
      if (bc != INT32_MAX) {
        const int64_t Ki = w.Kp[i];
        const i128 S = bsc - (i128)ct.A * kid - (i128)ct.p * Ki * (Ki - w.Sp[d]);
        bool propose = S > 0;
        if (REFINE && propose && w.Cp[bc] != bc) propose = false;
        if (propose) {
          const unsigned slot = atomicAdd(&sm.nprop, 1u);
          w.pi[slot] = i;
          w.pc[slot] = bc;
          w.pS[slot] = S;
          if (REFINE) w.stamp[i] = sv;
        }
      }
    }
    __syncthreads();
  }
}

// Commits of a local-moving sub-sweep; returns this thread's share of sum S.
template <typename WT>
__device__ i128 apply_moves(const Lvl<WT> &g, WS &w, const Ctl &ct, Shared &sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const unsigned np = sm.nprop;
  i128 acc = 0;
  for (unsigned m = warp; m < np; m += nw) {
    const int32_t i = w.pi[m], c = w.pc[m];
    if (lane == 0) {
      const int32_t d = w.Cp[i];
      const int64_t Ki = w.Kp[i];
      atomic_add_i64(&w.Sp[d], -Ki);
      atomic_add_i64(&w.Sp[c], Ki);
      w.Cp[i] = c;
      if (ct.dynamic) { w.ch[d] = 1; w.ch[c] = 1; }
      acc += w.pS[m];
    }
    for (int64_t e = g.off[i] + lane; e < g.off[i + 1]; e += 32) {
      const int32_t j = g.idx[e];
      if (w.proc[j]) w.proc[j] = 0;   // most are unprocessed already: spare the store
    }
  }
  __syncthreads();
  return acc;
}

// Commits of a refinement sub-sweep; returns this thread's count of moves.
__device__ int64_t apply_refine(WS &w, uint8_t sv, Shared &sm) {
  const unsigned np = sm.nprop;
  int64_t moved = 0;
  for (unsigned m = threadIdx.x; m < np; m += blockDim.x) {
    const int32_t i = w.pi[m], c = w.pc[m];
    if (w.stamp[c] == sv) continue;
    const int64_t Ki = w.Kp[i];
    atomic_add_i64(&w.Sp[i], -Ki);
    atomic_add_i64(&w.Sp[c], Ki);
    w.Cp[i] = c;
    moved++;
  }
  __syncthreads();
  return moved;
}

// Vertex list sorted by colour class (vertices of degree 0 left out).
template <typename WT>
__device__ void build_classes(const Lvl<WT> &g, WS &w, int log2S, Shared &sm) {
  const int S = 1 << log2S;
  for (int k = threadIdx.x; k < S; k += blockDim.x) sm.kcur[k] = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x)
    if (g.off[i + 1] > g.off[i]) atomicAdd(&sm.kcur[det_class((int32_t)i, log2S)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int k = 0; k < S; k++) { sm.koff[k] = run; run += sm.kcur[k]; sm.kcur[k] = sm.koff[k]; }
    sm.koff[S] = run;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x)
    if (g.off[i + 1] > g.off[i]) w.vl[atomicAdd(&sm.kcur[det_class((int32_t)i, log2S)], 1)] = (int32_t)i;
  __syncthreads();
}

// Alg. leidenlm; returns l_i, adds the migrations to *moves (thread 0).
template <typename WT>
__device__ int local_move(const Lvl<WT> &g, WS &w, const Ctl &ct, double tau, int max_iters, int64_t *moves,
                          int32_t *skeys, u64 *svals, Shared &sm) {
  const int S = 1 << ct.log2S;
  int li = 0;
  while (li < max_iters) {
    i128 acc = 0;
    for (int s = 0; s < S; s++) {
      decide<false>(g, w, ct, sm.koff[s], sm.koff[s + 1], 0, skeys, svals, sm);
      if (threadIdx.x == 0) *moves += sm.nprop;
      acc += apply_moves(g, w, ct, sm);
    }
    li++;
    const i128 tot = bsum128(acc, sm);
    if (threadIdx.x == 0) sm.stop = (ct.two_m == 0 || i128_to_double(tot) / ct.den <= tau) ? 1 : 0;
    __syncthreads();
    const int stop = sm.stop;
    __syncthreads();
    if (stop) break;
  }
  return li;
}

// Alg. leidenre: one sweep, one sub-sweep per colour class.
template <typename WT>
__device__ int64_t refine(const Lvl<WT> &g, WS &w, const Ctl &ct, int32_t *skeys, u64 *svals, Shared &sm) {
  const int S = 1 << ct.log2S;
  for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) w.stamp[i] = 0;
  __syncthreads();
  int64_t moved = 0;
  for (int s = 0; s < S; s++) {
    const uint8_t sv = (uint8_t)(s % 255 + 1);
    if (s > 0 && sv == 1) {
      for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) w.stamp[i] = 0;
      __syncthreads();
    }
    decide<true>(g, w, ct, sm.koff[s], sm.koff[s + 1], sv, skeys, svals, sm);
    moved += apply_refine(w, sv, sm);
  }
  return bsum64(moved, sm);
}

// Alg. leidensr (representative = smallest member), then C'_B = C' and the
// break of changed communities into singletons.
__device__ void subset_renumber_and_break(int64_t n, WS &w, Shared &sm) {
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) { w.rep[c] = INT_MAX; w.S2[c] = 0; w.ch2[c] = 0; }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) atomicMin(&w.rep[w.Cp[i]], (int32_t)i);
  __syncthreads();
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    const int32_t r = w.rep[c];
    if (r == INT_MAX) continue;
    w.S2[r] = w.Sp[c];
    w.ch2[r] = w.ch[c];
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) w.Cp[i] = w.rep[w.Cp[i]];
  __syncthreads();
  { int64_t *t = w.Sp; w.Sp = w.S2; w.S2 = t; }
  { uint8_t *t = w.ch; w.ch = w.ch2; w.ch2 = t; }
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t c = w.Cp[i];
    w.CB[i] = c;
    if (w.ch[c]) { w.Cp[i] = (int32_t)i; w.Sp[i] = w.Kp[i]; }
  }
  __syncthreads();
}

// Dense renumbering in increasing order of the old ID; returns the count.
__device__ int64_t renumber(int64_t n, WS &w, Shared &sm) {
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) w.flag[c] = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) w.flag[w.Cp[i]] = 1;
  __syncthreads();
  bscan<uint8_t>(w.flag, w.scn, n, sm);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) w.Cp[i] = (int32_t)w.scn[w.Cp[i]];
  const int64_t nc = w.scn[n];
  __syncthreads();
  return nc;
}

__device__ void lookup(int64_t N, WS &w) {
  for (int64_t v = threadIdx.x; v < N; v += blockDim.x) w.Ctop[v] = w.Cp[w.Ctop[v]];
  __syncthreads();
}

// Adds every entry of member rows of community c (warp-uniform member walk)
// to a table: K_{c -> d} for every community d, self-loops included.
template <typename WT>
__device__ void agg_rows(const Lvl<WT> &g, const WS &w, int64_t m0, int64_t m1, int64_t mstep, int32_t *keys,
                         u64 *vals, int lh, u64 *scr, u64 *err) {
  const int lane = threadIdx.x & 31;
  for (int64_t m = m0; m < m1; m += mstep) {
    const int32_t v = w.cv[m];
    const int64_t e0 = g.off[v], e1 = g.off[v + 1];
    for (int64_t xb = e0; xb < e1; xb += 32) {
      const int64_t e = xb + lane;
      const bool in = e < e1;
      const int32_t c = in ? w.Cp[g.idx[e]] : LEIDEN_EMPTY_KEY;
      const u64 wv = in ? (u64)(int64_t)g.w[e] : 0;
      u64 sum = 0;
      if (warp_combine((unsigned long long)(uint32_t)c, in, wv, &sum, scr)) tbl_add(keys, vals, lh, c, sum, err);
    }
  }
}

// Alg. leidenag: super-vertex graph of the nc communities of Cp (renumbered)
// into (off2, idx2, w2); K'' = its row sums into Kp.  Returns its nnz.
template <typename WT>
__device__ int64_t aggregate(const Lvl<WT> &g, WS &w, int64_t nc, int64_t *off2, int32_t *idx2, int64_t *w2,
                             int32_t *skeys_all, u64 *svals_all, Shared &sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // community vertex lists and total degrees
  for (int64_t c = threadIdx.x; c < nc; c += blockDim.x) { w.ccur[c] = 0; w.cdist[c] = 0; }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x) {
    const int32_t c = w.Cp[i];
    atomicAdd((u64 *)&w.ccur[c], 1ull);
    atomicAdd((u64 *)&w.cdist[c], (u64)(g.off[i + 1] - g.off[i]));
  }
  __syncthreads();
  bscan<int64_t>(w.ccur, w.coff, nc, sm);
  bscan<int64_t>(w.cdist, w.hoff, nc, sm);
  for (int64_t c = threadIdx.x; c < nc; c += blockDim.x) w.ccur[c] = w.coff[c];
  __syncthreads();
  for (int64_t i = threadIdx.x; i < g.n; i += blockDim.x)
    w.cv[atomicAdd((u64 *)&w.ccur[w.Cp[i]], 1ull)] = (int32_t)i;
  if (threadIdx.x == 0) sm.nlong = 0;
  __syncthreads();
  // short communities: one warp each, shared-memory table
  int32_t *keys = skeys_all + warp * SB_WARP_SLOTS;
  u64 *vals = svals_all + warp * SB_WARP_SLOTS;
  for (int64_t c = warp; c < nc; c += nw) {
    const int64_t td = w.hoff[c + 1] - w.hoff[c];
    const int64_t cap = td < nc ? td : nc;
    if (2 * cap > SB_WARP_SLOTS) {
      if (lane == 0) w.longl[atomicAdd(&sm.nlong, 1u)] = (int32_t)c;
      continue;
    }
    const int lh = log2_at_least(2 * cap);
    for (int s = lane; s < (1 << lh); s += 32) { keys[s] = LEIDEN_EMPTY_KEY; vals[s] = 0; }
    __syncwarp();
    agg_rows(g, w, w.coff[c], w.coff[c + 1], 1, keys, vals, lh, sm.wscr[warp], &sm.err);
    __syncwarp();
    int64_t pos = w.hoff[c], ksum = 0;
    for (int sb = 0; sb < (1 << lh); sb += 32) {
      const int s = sb + lane;
      const bool occ = s < (1 << lh) && keys[s] != LEIDEN_EMPTY_KEY;
      const unsigned m = __ballot_sync(FULL_MASK, occ);
      if (occ) {
        const int64_t at = pos + __popc(m & ((1u << lane) - 1u));
        w.hidx[at] = keys[s];
        w.hw[at] = (int64_t)vals[s];
        ksum += (int64_t)vals[s];
      }
      pos += __popc(m);
    }
    for (int o = 16; o; o >>= 1) ksum += shfl_xor_i64(ksum, o);
    if (lane == 0) { w.cdist[c] = pos - w.hoff[c]; w.Kp[c] = ksum; }
    __syncwarp();
  }
  __syncthreads();
  // long communities: the whole block each, table in global scratch
  const unsigned nlong = sm.nlong;
  for (unsigned t = 0; t < nlong; t++) {
    const int32_t c = w.longl[t];
    const int64_t td = w.hoff[c + 1] - w.hoff[c];
    const int64_t cap = td < nc ? td : nc;
    int lh = log2_at_least(2 * cap);
    if (lh > w.log2T) { if (threadIdx.x == 0) atomicOr(&sm.err, 32ull); lh = w.log2T; }
    for (int64_t s = threadIdx.x; s < ((int64_t)1 << lh); s += blockDim.x) {
      w.gkeys[s] = LEIDEN_EMPTY_KEY;
      w.gvals[s] = 0;
    }
    __syncthreads();
    agg_rows(g, w, w.coff[c] + warp, w.coff[c + 1], nw, w.gkeys, w.gvals, lh, sm.wscr[warp], &sm.err);
    if (threadIdx.x == 0) sm.long_n = 0;
    __syncthreads();
    int64_t ksum = 0;
    for (int64_t sb = 32 * warp; sb < ((int64_t)1 << lh); sb += 32 * (int64_t)nw) {
      const int64_t s = sb + lane;
      const bool occ = s < ((int64_t)1 << lh) && w.gkeys[s] != LEIDEN_EMPTY_KEY;
      const u64 at = warp_reserve((u64 *)&sm.long_n, occ);
      if (occ) {
        w.hidx[w.hoff[c] + (int64_t)at] = w.gkeys[s];
        w.hw[w.hoff[c] + (int64_t)at] = (int64_t)w.gvals[s];
        ksum += (int64_t)w.gvals[s];
      }
    }
    ksum = bsum64(ksum, sm);
    if (threadIdx.x == 0) { w.cdist[c] = sm.long_n; w.Kp[c] = ksum; }
    __syncthreads();
  }
  // compact into the next level
  bscan<int64_t>(w.cdist, off2, nc, sm);
  for (int64_t c = warp; c < nc; c += nw) {
    const int64_t src = w.hoff[c], dst = off2[c], k = w.cdist[c];
    for (int64_t x = lane; x < k; x += 32) { idx2[dst + x] = w.hidx[src + x]; w2[dst + x] = w.hw[src + x]; }
  }
  __syncthreads();
  return off2[nc];
}

// One pass on level graph g (Alg. leiden body).  Returns 1 to stop, 0 to go
// on with the aggregated graph in (off2, idx2, w2) of *nc vertices / *nnz2.
template <typename WT>
__device__ int pass(const Lvl<WT> &g, WS &w, const Ctl &ct, int lp, double tau, const SmallOpts &o, int64_t N,
                    int64_t *off2, int32_t *idx2, int64_t *w2, int64_t *nc_out, int64_t *nnz_out, SmallResult *res,
                    int32_t *skeys, u64 *svals, Shared &sm) {
  build_classes(g, w, ct.log2S, sm);
  int64_t moves = 0;
  const int li = local_move(g, w, ct, tau, o.max_iters, &moves, skeys, svals, sm);
  if (lp == 0) {
    int64_t k = 0;
    for (int64_t c = threadIdx.x; c < g.n; c += blockDim.x) k += w.ch[c] != 0;
    k = bsum64(k, sm);
    if (threadIdx.x == 0) res->changed0 = k;
  }
  subset_renumber_and_break(g.n, w, sm);
  const int64_t rmoves = refine(g, w, ct, skeys, svals, sm);
  if (threadIdx.x == 0 && lp < LEIDEN_STATS_PASSES) {
    res->passes = lp + 1;
    res->iters[lp] = li;
    res->nv[lp] = g.n;
    res->moves[lp] = moves;
    res->refine_moves[lp] = rmoves;
  }
  if (lp > 0 && li <= 1) return 1;
  const int64_t nc = renumber(g.n, w, sm);
  *nc_out = nc;
  if (nc == g.n) return 1;
  lookup(N, w);
  *nnz_out = aggregate(g, w, nc, off2, idx2, w2, skeys, svals, sm);
  return 0;
}

// Checks of one job's inputs; returns a LEIDEN_ code.
__device__ int check_job(const SmallJob &j, Shared &sm) {
  if (threadIdx.x == 0) sm.err = 0;
  __syncthreads();
  const int64_t n = j.n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t a = j.off[i], b = j.off[i + 1];
    if (a > b || a < 0 || b > j.nnz) atomicOr(&sm.err, 1ull);
  }
  if (threadIdx.x == 0 && (j.off[0] != 0 || j.off[n] != j.nnz)) atomicOr(&sm.err, 1ull);
  for (int64_t e = threadIdx.x; e < j.nnz; e += blockDim.x)
    if (j.idx[e] < 0 || j.idx[e] >= n || j.w[e] <= 0) atomicOr(&sm.err, 1ull);
  if (j.mode != LEIDEN_STATIC) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
      if (j.prior[i] < 0 || j.prior[i] >= n) atomicOr(&sm.err, 1ull);
    for (int64_t k = threadIdx.x; k < j.nd + j.ni; k += blockDim.x) {
      const bool del = k < j.nd;
      const int64_t x = del ? k : k - j.nd;
      const int32_t u = del ? j.ds[x] : j.is[x], v = del ? j.dd[x] : j.id[x];
      const int32_t wt = del ? j.dw[x] : j.iw[x];
      if (u < 0 || u >= n || v < 0 || v >= n || u == v || wt <= 0) atomicOr(&sm.err, 1ull);
    }
  }
  __syncthreads();
  const int rc = sm.err ? LEIDEN_EINVAL : LEIDEN_OK;
  __syncthreads();
  return rc;
}

// Alg. delta inside one block: the affected vertices (w.flag, the range of
// the first pass; they start unprocessed), with w.ch2 as delta-E (vertices
// whose neighbours are affected) and w.stamp as delta-C (communities whose
// members are affected).  Deletions inside a community mark both ends and the
// community; for each source of insertions, the best community c* != its own
// by Eq. 2 with K_{i->c} the inserted weight towards c and K_{i->d} = 0 (ties
// to the smallest c) marks the source and c*.  K and Sigma are those of G^t
// and C^{t-1} (w.Kp, w.Sp).  Batches of the persistent path are small: each
// source's insertions are grouped by scanning the batch.
__device__ void mark_ds(const SmallJob &j, WS &w, const Ctl &ct, Shared &sm) {
  const int64_t N = j.n;
  uint8_t *aff = w.flag, *dE = w.ch2, *dC = w.stamp;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) { aff[i] = 0; dE[i] = 0; dC[i] = 0; }
  __syncthreads();
  for (int64_t k = threadIdx.x; k < j.nd; k += blockDim.x) {
    const int32_t u = j.ds[k], v = j.dd[k];
    const int32_t c = j.prior[u];
    if (c != j.prior[v]) continue;
    aff[u] = 1; dE[u] = 1;
    aff[v] = 1; dE[v] = 1;
    dC[c] = 1;
  }
  // directed insertion entries x in [0, 2 ni): (is, id) then (id, is)
  const int64_t E = 2 * j.ni;
  auto src = [&](int64_t x) { return x < j.ni ? j.is[x] : j.id[x - j.ni]; };
  auto dst = [&](int64_t x) { return x < j.ni ? j.id[x] : j.is[x - j.ni]; };
  auto wt = [&](int64_t x) { return (int64_t)(x < j.ni ? j.iw[x] : j.iw[x - j.ni]); };
  for (int64_t x = threadIdx.x; x < E; x += blockDim.x) {
    const int32_t u = src(x);
    bool first = true;
    for (int64_t y = 0; y < x && first; y++) first = src(y) != u;
    if (!first) continue;
    const int32_t d = j.prior[u];
    const int64_t Ki = w.Kp[u];
    int32_t best = INT32_MAX;
    i128 bS = 0;
    for (int64_t y = x; y < E; y++) {
      if (src(y) != u) continue;
      const int32_t c = j.prior[dst(y)];
      if (c == d) continue;
      bool seen = false;
      for (int64_t z = x; z < y && !seen; z++) seen = src(z) == u && j.prior[dst(z)] == c;
      if (seen) continue;
      int64_t h = 0;
      for (int64_t z = y; z < E; z++)
        if (src(z) == u && j.prior[dst(z)] == c) h += wt(z);
      const i128 S = (i128)ct.A * h - (i128)ct.p * Ki * (Ki + w.Sp[c] - w.Sp[d]);
      if (best == INT32_MAX || S > bS || (S == bS && c < best)) { bS = S; best = c; }
    }
    if (best != INT32_MAX) {
      aff[u] = 1;
      dE[u] = 1;
      dC[best] = 1;
    }
  }
  __syncthreads();
  // expansion: members of delta-C communities and neighbours of delta-E vertices
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    if (dC[j.prior[i]]) aff[i] = 1;
    if (dE[i])
      for (int64_t e = j.off[i]; e < j.off[i + 1]; e++) aff[j.idx[e]] = 1;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) w.proc[i] = aff[i] ? 0 : 1;
  __syncthreads();
}

// The whole of Alg. leiden for one job.
__device__ void run_job(const SmallJob &j, const SmallOpts &o, SmallResult *res, int32_t *skeys, u64 *svals,
                        Shared &sm) {
  const int64_t N = j.n;
  if (threadIdx.x == 0) {
    res->status = LEIDEN_OK;
    res->passes = 0;
    res->affected0 = 0;
    res->changed0 = 0;
  }
  int rc = check_job(j, sm);
  if (rc) {
    if (threadIdx.x == 0) res->status = rc;
    return;
  }
  WS w;
  carve_ws(j.ws, N, j.nnz, w);
  const Lvl<int32_t> g0{N, j.off, j.idx, j.w};
  // K = row sums of G^t; 2m = their total
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t i = warp; i < N; i += nw) {
    int64_t k = 0;
    for (int64_t e = j.off[i] + lane; e < j.off[i + 1]; e += 32) k += (int64_t)j.w[e];
    for (int o2 = 16; o2; o2 >>= 1) k += shfl_xor_i64(k, o2);
    if (lane == 0) w.Kp[i] = k;
  }
  __syncthreads();
  int64_t two_m = 0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) two_m += w.Kp[i];
  two_m = bsum64(two_m, sm);
  if (two_m < 0 || two_m >= ((int64_t)1 << 40)) {
    if (threadIdx.x == 0) res->status = LEIDEN_EOVERFLOW;
    return;
  }
  Ctl ct;
  ct.p = o.p;
  ct.q = o.q;
  ct.two_m = two_m;
  ct.A = two_m * o.q;
  ct.den = (double)two_m * (double)two_m * 0.5 * (double)o.q;
  ct.log2S = o.log2S;
  const bool upd = j.mode != LEIDEN_STATIC;
  ct.dynamic = upd ? 1 : 0;
  ct.in_range = nullptr;
  // initial state (Alg. leiden / update / naive / frontier)
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    w.Ctop[i] = (int32_t)i;
    w.Cp[i] = upd ? j.prior[i] : (int32_t)i;
    w.Sp[i] = upd ? 0 : w.Kp[i];
    w.ch[i] = upd ? (o.refine_all_first_pass ? 1 : 0) : 1;
    w.proc[i] = (upd && j.mode == LEIDEN_DF) ? 1 : 0;
  }
  __syncthreads();
  if (upd) {
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
      if (w.Kp[i]) atomic_add_i64(&w.Sp[w.Cp[i]], w.Kp[i]);
    for (int64_t k = threadIdx.x; k < j.nd + j.ni; k += blockDim.x) {
      const bool del = k < j.nd;
      const int64_t x = del ? k : k - j.nd;
      const int32_t u = del ? j.ds[x] : j.is[x], v = del ? j.dd[x] : j.id[x];
      const bool same = j.prior[u] == j.prior[v];
      if (same && !o.refine_all_first_pass) w.ch[j.prior[u]] = 1;          // changedCommunities
      if (j.mode == LEIDEN_DF && same == del) { w.proc[u] = 0; w.proc[v] = 0; }  // Alg. frontier
    }
    __syncthreads();
    if (j.mode == LEIDEN_DS) {
      mark_ds(j, w, ct, sm);
      ct.in_range = w.flag;
    }
    int64_t a = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) a += w.proc[i] == 0;
    a = bsum64(a, sm);
    if (threadIdx.x == 0) res->affected0 = a;
  } else if (threadIdx.x == 0) {
    res->affected0 = N;
  }
  __syncthreads();

  double tau = o.tol;
  int cur = -1;  // -1: the input graph; 0 / 1: level buffers A / B
  int64_t nv = N, nnz_cur = j.nnz;
  int lp;
  for (lp = 0; lp < o.max_passes; lp++) {
    if (threadIdx.x == 0 && lp < LEIDEN_STATS_PASSES) res->nnz[lp] = nnz_cur;
    const int dst = cur < 0 ? 0 : 1 - cur;
    int64_t *off2 = dst == 0 ? w.offA : w.offB;
    int32_t *idx2 = dst == 0 ? w.idxA : w.idxB;
    int64_t *w2 = dst == 0 ? w.wA : w.wB;
    int64_t nc = 0, nnz2 = 0;
    int r;
    if (cur < 0) {
      r = pass(g0, w, ct, lp, tau, o, N, off2, idx2, w2, &nc, &nnz2, res, skeys, svals, sm);
    } else {
      const Lvl<int64_t> gl{nv, cur == 0 ? w.offA : w.offB, cur == 0 ? w.idxA : w.idxB, cur == 0 ? w.wA : w.wB};
      r = pass(gl, w, ct, lp, tau, o, N, off2, idx2, w2, &nc, &nnz2, res, skeys, svals, sm);
    }
    ct.dynamic = 0;
    ct.in_range = nullptr;
    if (r == 1) break;
    cur = dst;
    nv = nc;
    nnz_cur = nnz2;
    for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) {
      w.Sp[i] = w.Kp[i];
      w.Cp[i] = (int32_t)i;
      w.proc[i] = 0;
      w.ch[i] = 1;
    }
    __syncthreads();
    tau /= o.tol_drop;
  }
  lookup(N, w);
  // canonical labels
  for (int64_t c = threadIdx.x; c < N; c += blockDim.x) { w.rep[c] = INT_MAX; w.flag[c] = 0; }
  __syncthreads();
  for (int64_t v = threadIdx.x; v < N; v += blockDim.x) atomicMin(&w.rep[w.Ctop[v]], (int32_t)v);
  __syncthreads();
  for (int64_t c = threadIdx.x; c < N; c += blockDim.x)
    if (w.rep[c] != INT_MAX) w.flag[w.rep[c]] = 1;
  __syncthreads();
  bscan<uint8_t>(w.flag, w.scn, N, sm);
  for (int64_t v = threadIdx.x; v < N; v += blockDim.x) j.out[v] = (int32_t)w.scn[w.rep[w.Ctop[v]]];
  __syncthreads();
  // Eq. 1 terms of the returned membership on the input graph
  for (int64_t c = threadIdx.x; c < N; c += blockDim.x) w.S2[c] = 0;
  __syncthreads();
  int64_t inside = 0;
  for (int64_t i = warp; i < N; i += nw) {
    const int32_t ci = j.out[i];
    int64_t k = 0;
    for (int64_t e = j.off[i] + lane; e < j.off[i + 1]; e += 32) {
      const int64_t x = (int64_t)j.w[e];
      k += x;
      if (j.out[j.idx[e]] == ci) inside += x;
    }
    for (int o2 = 16; o2; o2 >>= 1) k += shfl_xor_i64(k, o2);
    if (lane == 0 && k) atomic_add_i64(&w.S2[ci], k);
  }
  inside = bsum64(inside, sm);
  i128 sq = 0;
  for (int64_t c = threadIdx.x; c < N; c += blockDim.x) sq += (i128)w.S2[c] * w.S2[c];
  sq = bsum128(sq, sm);
  if (threadIdx.x == 0) {
    res->inside = inside;
    res->two_m = two_m;
    res->sq_lo = (u64)sq;
    res->sq_hi = (u64)(sq >> 64);
    if (sm.err) res->status = LEIDEN_ECUDA;
  }
  __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(512) small_leiden_k(SmallHeader *hdr, const SmallJob *jobs, SmallOpts o,
                                                       SmallResult *results) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Shared sm;
  const int nw = blockDim.x >> 5;
  u64 *svals = reinterpret_cast<u64 *>(dsm);
  int32_t *skeys = reinterpret_cast<int32_t *>(svals + (size_t)nw * SB_WARP_SLOTS);
  const int count = hdr->count;
  for (;;) {
    if (threadIdx.x == 0) sm.job = (int)atomicAdd(&hdr->next, 1u);
    __syncthreads();
    const int k = sm.job;
    __syncthreads();
    if (k >= count) break;
    if (threadIdx.x == 0) sm.err = 0;
    __syncthreads();
    run_job(jobs[k], o, &results[jobs[k].result], skeys, svals, sm);
  }
}

size_t small_dyn_smem(int threads) { return (size_t)(threads / 32) * SB_WARP_SLOTS * (sizeof(u64) + sizeof(int32_t)); }

}  // namespace lk
