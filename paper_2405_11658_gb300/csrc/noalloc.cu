// noalloc.cu -- modularity without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// modularity value: code running under a memory budget that forbids new
// allocations, plugins handed a stream but no allocator, or latency-critical
// loops that cannot afford the implicit device synchronisation cudaMalloc and
// cudaFree bring.  leiden_modularity_noalloc serves them: it needs no
// leiden_ctx (whose creation allocates the workspace) and keeps its scratch --
// the per-community totals and the accumulators -- in one fixed array that
// lives in this library's device image.  Every GPU that loads the library
// holds that array until the process exits.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "leiden.h"

namespace {

// Scratch of the allocation-free entry point: LEIDEN_NOALLOC_MAX_N int64
// per-community totals, then 16 words for accumulators and the error flag.
constexpr int64_t kWords = (int64_t)LEIDEN_NOALLOC_MAX_N + 16;
__device__ __align__(256) unsigned long long g_noalloc_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};

// The device address of the scratch array on the current device.  In host
// code the array's name is only a host-side stand-in, so the address comes
// from cudaGetSymbolAddress, once per device, with that device current.
int scratch_for_current_device(unsigned long long **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LEIDEN_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LEIDEN_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LEIDEN_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
  }
  *out = g_scratch_ptr[dev];
  return LEIDEN_OK;
}

}  // namespace

extern "C" int leiden_modularity_noalloc(const leiden_csr *g, const int32_t *membership, double gamma,
                                         void *cuda_stream, double *q_out) {
  if (!g || !q_out || g->n < 0 || g->nnz < 0) return LEIDEN_EINVAL;
  if (g->n > LEIDEN_NOALLOC_MAX_N) return LEIDEN_ENOMEM;  // beyond the fixed scratch
  // the u64 accumulators cannot wrap while nnz <= 2^32 (every weight < 2^31)
  if (g->nnz > ((int64_t)1 << 32)) return LEIDEN_EOVERFLOW;
  if (!g->off || (g->n > 0 && !membership) || (g->nnz > 0 && (!g->idx || !g->w))) return LEIDEN_EINVAL;
  // gamma = p / q exactly, q = 2^20 before reduction
  const double scaled = gamma * 1048576.0;
  if (!(gamma > 0.0) || scaled > 9.0e15) return LEIDEN_EINVAL;
  int64_t p = (int64_t)scaled;
  if ((double)p != scaled) return LEIDEN_EINVAL;
  int64_t q = 1048576;
  {
    int64_t a = p, b = q;
    while (b) { const int64_t t = a % b; a = b; b = t; }
    p /= a;
    q /= a;
  }
  unsigned long long *scr = nullptr;
  int rc = scratch_for_current_device(&scr);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int64_t *sig = reinterpret_cast<int64_t *>(scr);
  unsigned long long *acc = scr + LEIDEN_NOALLOC_MAX_N;  // [0..3] terms, [8] error flag
  unsigned long long h[9] = {0};
  // The array keeps the previous call's contents: clear what must start at 0.
  // Validate the graph and the labels, and read the verdict on the host,
  // before any kernel indexes by them.
  cudaMemsetAsync(acc + 8, 0, sizeof(unsigned long long), s);
  lk::launch_check_graph(g->n, g->nnz, g->off, g->idx, g->w, acc + 8, s);
  lk::launch_check_range(membership, g->n, g->n, acc + 8, s);
  cudaMemcpyAsync(&h[8], acc + 8, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return LEIDEN_ECUDA;
  if (h[8]) return LEIDEN_EINVAL;
  // The terms kernels test every index themselves as well (a bad one is
  // skipped and flagged), so no access depends on the order above.
  lk::GraphView<int32_t> gv{g->n, g->off, g->idx, g->w};
  lk::launch_modularity_terms(gv, g->nnz, membership, sig, acc, acc + 8, s);  // zeroes sig[0..n), acc[0..3]
  cudaMemcpyAsync(h, acc, 9 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return LEIDEN_ECUDA;
  if (h[8]) return LEIDEN_EINVAL;
  const int64_t inside = (int64_t)h[0];
  const i128 sq = (i128)(((unsigned __int128)h[2] << 64) | (unsigned __int128)h[1]);
  const int64_t two_m = (int64_t)h[3];
  if (two_m < 0 || two_m >= ((int64_t)1 << 40)) return LEIDEN_EOVERFLOW;
  const i128 num = (i128)q * two_m * inside - (i128)p * sq;
  *q_out = two_m == 0 ? 0.0 : (double)num / ((double)two_m * (double)two_m * (double)q);
  return LEIDEN_OK;
}
