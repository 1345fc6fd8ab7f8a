// scan.cu -- exclusive prefix sums (reduce-then-scan, three launches).
//
// out[i] = in[0] + ... + in[i-1] for i in [0, n], so out[n] is the total.
// Used for the exclusive scans of the aggregation phase (Alg. leidenag:
// community-vertex offsets and super-vertex offsets), the dense renumbering of
// communities, the canonical relabelling and the batch application.
#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "internal.h"

namespace lk {

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (once per
// kernel and size; the attribute outlives the call, so it is set only when
// the requested size grows).
void ensure_smem(const void *func, size_t bytes) {
  if (bytes <= 32 * 1024) return;  // leaves room for static shared memory
  static std::mutex mu;
  static std::unordered_map<const void *, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  size_t &have = done[func];
  if (have >= bytes) return;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    have = bytes;
}

int64_t resident_blocks(const void *func, int threads, size_t smem, int sms) {
  struct Key {
    const void *f;
    int t;
    size_t m;
    bool operator==(const Key &o) const { return f == o.f && t == o.t && m == o.m; }
  };
  struct Hash {
    size_t operator()(const Key &k) const {
      return std::hash<const void *>()(k.f) ^ ((size_t)k.t << 20) ^ (k.m << 1);
    }
  };
  static std::mutex mu;
  static std::unordered_map<Key, int, Hash> per_sm;
  int nb = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = per_sm.find(Key{func, threads, smem});
    if (it != per_sm.end()) {
      nb = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, func, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        nb = 0;
      }
      if (nb < 1) nb = 1;
      per_sm[Key{func, threads, smem}] = nb;
    }
  }
  return (int64_t)nb * sms;
}

static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename TI>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_reduce(const TI *in, int64_t n, int64_t *partial) {
  __shared__ int64_t sbuf[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) s += (int64_t)in[i];
  }
  s = block_sum_i64(s, sbuf);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Single block: exclusive scan of partial[0..nb) in place; writes the total to
// *total_out.
__global__ void __launch_bounds__(1024) scan_partials(int64_t *partial, int64_t nb, int64_t *total_out) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < nb; base += 1024) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? partial[i] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = shfl_i64(x, (lane - o) & 31);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t t = warp_tot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = shfl_i64(t, (lane - o) & 31);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    int64_t warp_prefix = warp ? warp_tot[warp - 1] : 0;
    int64_t carry = carry_s;
    if (i < nb) partial[i] = carry + warp_prefix + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + warp_tot[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry_s;
}

template <typename TI>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_apply(const TI *in, int64_t n, const int64_t *partial, int64_t *out) {
  __shared__ int64_t warp_tot[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t i = base + k;
    v[k] = i < n ? (int64_t)in[i] : 0;
    s += v[k];
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = shfl_i64(x, (lane - o) & 31);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  int64_t wp = 0;
  for (int k = 0; k < warp; k++) wp += warp_tot[k];
  int64_t run = partial[blockIdx.x] + wp + x - s;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

template <typename TI>
void exclusive_scan(const TI *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    return;
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  LK_COUNTED scan_tile_reduce<TI><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, tmp);
  LK_COUNTED scan_partials<<<1, 1024, 0, s>>>(tmp, nb, out + n);
  LK_COUNTED scan_tile_apply<TI><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, tmp, out);
}

template void exclusive_scan<uint8_t>(const uint8_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template void exclusive_scan<int32_t>(const int32_t *, int64_t *, int64_t, int64_t *, cudaStream_t);
template void exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *, cudaStream_t);

}  // namespace lk
