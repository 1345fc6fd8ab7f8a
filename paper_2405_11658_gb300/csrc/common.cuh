// common.cuh -- device-side helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

typedef __int128 i128;
typedef unsigned long long u64;

#define LEIDEN_EMPTY_KEY (-1)
#define FULL_MASK 0xffffffffu

namespace lk {

// Value type of the decide kernels' hashtables.  The 64-bit score path is
// taken only when 4 (2m)^2 max(p, q) < 2^62, so 2m < 2^31 and every summed
// K_{i->c} (at most K_i <= 2m) fits 32 bits: those tables hold 8-byte slots
// instead of 12.
template <typename ST> struct TableVal { typedef u64 type; };
template <> struct TableVal<int64_t> { typedef uint32_t type; };

__device__ __forceinline__ void add_val(u64 *p, u64 w) { atomicAdd(p, w); }
__device__ __forceinline__ void add_val(uint32_t *p, u64 w) { atomicAdd((unsigned *)p, (unsigned)w); }

// Multiplicative hash of a community ID; the top bits index the table.
__device__ __forceinline__ uint32_t hash32(int32_t c) {
  return (uint32_t)c * 0x9E3779B1u;
}

// DET colour class: top log2(S) bits of (uint32)(i * 2654435761).
__host__ __device__ __forceinline__ int det_class(int32_t i, int log2S) {
  if (log2S == 0) return 0;
  uint32_t h = (uint32_t)i * 2654435761u;
  return (int)(h >> (32 - log2S));
}

__device__ __forceinline__ int64_t shfl_xor_i64(int64_t v, int off) {
  return (int64_t)__shfl_xor_sync(FULL_MASK, (long long)v, off);
}
__device__ __forceinline__ int64_t shfl_i64(int64_t v, int src) {
  return (int64_t)__shfl_sync(FULL_MASK, (long long)v, src);
}
__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int off) {
  long long lo = (long long)(u64)v;
  long long hi = (long long)(v >> 64);
  lo = __shfl_xor_sync(FULL_MASK, lo, off);
  hi = __shfl_xor_sync(FULL_MASK, hi, off);
  return ((i128)hi << 64) | (i128)(u64)lo;
}
__device__ __forceinline__ i128 shfl_i128(i128 v, int src) {
  long long lo = (long long)(u64)v;
  long long hi = (long long)(v >> 64);
  lo = __shfl_sync(FULL_MASK, lo, src);
  hi = __shfl_sync(FULL_MASK, hi, src);
  return ((i128)hi << 64) | (i128)(u64)lo;
}
template <typename T> __device__ __forceinline__ T shfl_xor_any(T v, int off);
template <> __device__ __forceinline__ int64_t shfl_xor_any<int64_t>(int64_t v, int off) { return shfl_xor_i64(v, off); }
template <> __device__ __forceinline__ i128 shfl_xor_any<i128>(i128 v, int off) { return shfl_xor_i128(v, off); }
template <typename T> __device__ __forceinline__ T shfl_any(T v, int src);
template <> __device__ __forceinline__ int64_t shfl_any<int64_t>(int64_t v, int src) { return shfl_i64(v, src); }
template <> __device__ __forceinline__ i128 shfl_any<i128>(i128 v, int src) { return shfl_i128(v, src); }

// Exact signed 128-bit accumulation into two 64-bit words with two atomics:
// the word that wraps is detected by the adder that wrapped it, so every carry
// is counted exactly once and the pair holds the sum modulo 2^128.
__device__ __forceinline__ void atomic_add_i128(u64 *acc /* [lo, hi] */, i128 x) {
  u64 lo = (u64)x;
  u64 hi = (u64)(x >> 64);
  u64 old = atomicAdd(&acc[0], lo);
  u64 carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(&acc[1], hi + carry);
}

__device__ __forceinline__ void atomic_add_i64(int64_t *p, int64_t v) {
  atomicAdd((u64 *)p, (u64)v);
}

// ASYNC refinement (Alg. leidenre with the paper's in-place updates): singleton
// i leaves its own community for c.  i leaves only while still isolated
// (Sigma'[i] = K'[i]); its total then holds REFINE_LEFT, far below any sum of
// degrees, for the rest of the phase, so a vertex about to join i's community
// sees a negative total and undoes its step -- however many other joiners are
// adding and undoing at the same moment.  (Marking with 0 is not enough: a
// second joiner's add, not yet undone, can hide it from a third, which would
// then join a community whose own vertex has left.)  Returns true once i is in
// c; the caller writes C'[i].  A sub-community never loses the vertex it is
// named after, so every member stays connected to it.
static constexpr int64_t REFINE_LEFT = INT64_MIN / 2;
// Sigma'[c] as a score reads it: a community whose own vertex has left
// (ASYNC refinement) counts as empty, and its marker never enters a product.
__device__ __forceinline__ int64_t sigma_for_score(const int64_t *Sig, int32_t c) {
  const int64_t v = Sig[c];
  return v < 0 ? 0 : v;
}
__device__ __forceinline__ bool refine_join_async(int64_t *Sig, int32_t i, int64_t Ki, int32_t c) {
  if ((int64_t)atomicCAS((unsigned long long *)&Sig[i], (unsigned long long)Ki,
                         (unsigned long long)REFINE_LEFT) != Ki)
    return false;
  const int64_t prev = (int64_t)atomicAdd((unsigned long long *)&Sig[c], (unsigned long long)Ki);
  if (prev < 0) {  // c's own vertex has left: undo both steps and stay
    atomic_add_i64(&Sig[c], -Ki);
    atomic_add_i64(&Sig[i], Ki - REFINE_LEFT);
    return false;
  }
  return true;
}

// Warp-aggregated reservation of `want` (0/1 per lane) slots in a counter;
// returns this lane's slot (valid where want != 0).  Whole warp must call.
__device__ __forceinline__ u64 warp_reserve(u64 *counter, bool want) {
  unsigned m = __ballot_sync(FULL_MASK, want);
  if (!m) return 0;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  u64 base = 0;
  if (lane == leader) base = atomicAdd(counter, (u64)__popc(m));
  base = __shfl_sync(FULL_MASK, base, leader);
  return base + __popc(m & ((1u << lane) - 1u));
}

// Combines equal keys across the active lanes of a warp before they reach a
// hashtable: returns true in exactly one lane per distinct key (the lowest),
// with *sum = the total weight of that key over the active lanes.  Turns a
// warp's worth of same-address atomics (e.g. the internal edges of a
// community, which all hash to one slot) into a single one.  The whole warp
// must call; `scratch` is 32 words of this warp's shared memory.
__device__ __forceinline__ bool warp_combine(unsigned long long key, bool active, u64 w, u64 *sum,
                                             u64 *scratch) {
  const unsigned act = __ballot_sync(FULL_MASK, active);
  const int lane = threadIdx.x & 31;
  bool lead = false;
  if (active) {
    const unsigned peers = __match_any_sync(act, key);
    scratch[lane] = w;
    __syncwarp(act);
    if (lane == __ffs(peers) - 1) {
      u64 s = 0;
      for (unsigned m = peers; m; m &= m - 1) s += scratch[__ffs(m) - 1];
      *sum = s;
      lead = true;
    }
  }
  __syncwarp();
  return lead;
}

// Block-wide sum of an i128 (every thread of the block must call); the result
// is valid in thread 0.  Uses 32 * 16 bytes of the given shared buffer.
__device__ __forceinline__ i128 block_sum_i128(i128 v, i128 *sbuf) {
  for (int o = 16; o; o >>= 1) v += shfl_xor_i128(v, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sbuf[warp] = v;
  __syncthreads();
  i128 r = 0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; k++) r += sbuf[k];
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ int64_t block_sum_i64(int64_t v, int64_t *sbuf) {
  for (int o = 16; o; o >>= 1) v += shfl_xor_i64(v, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sbuf[warp] = v;
  __syncthreads();
  int64_t r = 0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; k++) r += sbuf[k];
  }
  __syncthreads();
  return r;
}

}  // namespace lk
