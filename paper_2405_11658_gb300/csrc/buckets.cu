// buckets.cu -- vertex (or community) lists per (colour class, degree tier).
//
// key(v) = class(v) * ntiers + tier(deg(v)), deg(v) = off[v+1] - off[v].
// Counting sort in three steps: a per-block shared-memory histogram written as
// a [key][block] matrix, an exclusive scan of that matrix, and a scatter that
// starts every (key, block) run at its scanned offset.  The result is stored
// key-major; koff[key] .. koff[key+1] delimit each bucket.
#include "common.cuh"
#include "internal.h"

namespace lk {

static constexpr int BK_THREADS = 256;
static constexpr int BK_CHUNK = 8192;  // vertices per block

struct TierMax {
  int n;
  int64_t maxdeg[MAX_TIERS];
};

__device__ __forceinline__ int tier_of(int64_t deg, const TierMax &tm) {
  for (int t = 0; t < tm.n - 1; t++)
    if (deg <= tm.maxdeg[t]) return t;
  return tm.n - 1;
}

__global__ void __launch_bounds__(BK_THREADS) bucket_count_k(const int64_t *off, int64_t n, int log2S,
                                                             TierMax tm, int nkeys, int32_t *blockhist) {
  extern __shared__ int32_t hist[];
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * BK_CHUNK;
  for (int64_t v = base + threadIdx.x; v < n && v < base + BK_CHUNK; v += blockDim.x) {
    const int key = det_class((int32_t)v, log2S) * tm.n + tier_of(off[v + 1] - off[v], tm);
    atomicAdd(&hist[key], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x)
    blockhist[(int64_t)k * gridDim.x + blockIdx.x] = hist[k];
}

__global__ void __launch_bounds__(BK_THREADS) bucket_scatter_k(const int64_t *off, int64_t n, int log2S,
                                                               TierMax tm, int nkeys,
                                                               const int64_t *scanned, int32_t *list) {
  extern __shared__ int64_t cur[];
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x)
    cur[k] = scanned[(int64_t)k * gridDim.x + blockIdx.x];
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * BK_CHUNK;
  for (int64_t v = base + threadIdx.x; v < n && v < base + BK_CHUNK; v += blockDim.x) {
    const int key = det_class((int32_t)v, log2S) * tm.n + tier_of(off[v + 1] - off[v], tm);
    const int64_t pos = (int64_t)atomicAdd((u64 *)&cur[key], 1ull);
    list[pos] = (int32_t)v;
  }
}

__global__ void bucket_koff_k(const int64_t *scanned, int nkeys, int64_t nblocks, int64_t *koff) {
  for (int k = threadIdx.x; k <= nkeys; k += blockDim.x) koff[k] = scanned[(int64_t)k * nblocks];
}

int64_t bucket_blockhist_elems(int64_t n, int nkeys) {
  const int64_t nb = (n + BK_CHUNK - 1) / BK_CHUNK;
  return (nb < 1 ? 1 : nb) * (int64_t)nkeys + 1;
}

void launch_buckets(const int64_t *off, int64_t n, int log2S, const TierTable &tt, int32_t *list,
                    int32_t *blockhist, int64_t *scanned, int64_t *koff_dev, int64_t *scan_tmp,
                    cudaStream_t s) {
  TierMax tm{};
  tm.n = tt.ntiers;
  for (int t = 0; t < tt.ntiers; t++) tm.maxdeg[t] = tt.t[t].maxdeg;
  const int nkeys = (1 << log2S) * tt.ntiers;
  int64_t nb = (n + BK_CHUNK - 1) / BK_CHUNK;
  if (nb < 1) nb = 1;
  LK_COUNTED bucket_count_k<<<(unsigned)nb, BK_THREADS, nkeys * sizeof(int32_t), s>>>(off, n, log2S, tm, nkeys,
                                                                          blockhist);
  exclusive_scan<int32_t>(blockhist, scanned, nb * nkeys, scan_tmp, s);
  LK_COUNTED bucket_scatter_k<<<(unsigned)nb, BK_THREADS, nkeys * sizeof(int64_t), s>>>(off, n, log2S, tm, nkeys,
                                                                            scanned, list);
  LK_COUNTED bucket_koff_k<<<1, 256, 0, s>>>(scanned, nkeys, nb, koff_dev);
}

}  // namespace lk
