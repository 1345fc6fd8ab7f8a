// batch.cu -- host driver of the persistent many-graph kernel
// (leiden_batch_*): workspace carving, job descriptors, and the CUDA graph
// that uploads the descriptors, runs the kernel and downloads the results in
// one launch.
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.h"
#include "leiden.h"
#include "small.h"

using namespace lk;

struct leiden_batch {
  cudaStream_t st = nullptr;     // the caller's stream: every run is ordered on it
  cudaStream_t cap = nullptr;    // private stream the CUDA graph is captured on
  int device = 0, sms = 152, threads = 512, bps = 1;
  int32_t max_graphs = 0;
  int64_t max_n = 0, max_nnz = 0;
  char *arena = nullptr;
  int64_t arena_bytes = 0;
  char *d_desc = nullptr;        // SmallHeader, then SmallJob[max_graphs]
  SmallResult *d_res = nullptr;
  char *h_desc = nullptr;        // pinned staging of d_desc
  SmallResult *h_res = nullptr;  // pinned copy of d_res
  size_t desc_bytes = 0, res_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  SmallOpts captured{};          // kernel argument baked into the graph
  bool have_exec = false;
};

namespace {

void release(leiden_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->arena) cudaFree(b->arena);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_res) cudaFree(b->d_res);
  if (b->h_desc) cudaFreeHost(b->h_desc);
  if (b->h_res) cudaFreeHost(b->h_res);
  if (b->cap) cudaStreamDestroy(b->cap);
}

int opts_to_small(const leiden_opts *o, SmallOpts *so) {
  if (!o || o->sched != LEIDEN_DET) return LEIDEN_EINVAL;
  if (o->max_iters < 1 || o->max_passes < 1 || !(o->tol >= 0.0) || !(o->tol_drop > 0.0)) return LEIDEN_EINVAL;
  if (o->reserved[0] || o->reserved[1] || o->reserved[2]) return LEIDEN_EINVAL;
  const int S = o->det_subsets;
  if (S < 1 || S > 256 || (S & (S - 1))) return LEIDEN_EINVAL;
  int k = 0;
  while ((1 << k) < S) k++;
  const double scaled = o->gamma * 1048576.0;
  if (!(o->gamma > 0.0) || scaled > 9.0e15) return LEIDEN_EINVAL;
  int64_t p = (int64_t)scaled;
  if ((double)p != scaled) return LEIDEN_EINVAL;
  int64_t q = 1048576, a = p, bb = q;
  while (bb) { const int64_t t = a % bb; a = bb; bb = t; }
  so->p = p / a;
  so->q = q / a;
  so->tol = o->tol;
  so->tol_drop = o->tol_drop;
  so->max_iters = o->max_iters;
  so->max_passes = o->max_passes;
  so->log2S = k;
  so->refine_all_first_pass = o->refine_all_first_pass ? 1 : 0;
  return LEIDEN_OK;
}

int check_item(const leiden_batch_item &it) {
  const leiden_csr &g = it.g;
  if (g.n < 0 || g.nnz < 0 || g.n >= INT32_MAX || !g.off) return LEIDEN_EINVAL;
  if (g.nnz > 0 && (!g.idx || !g.w)) return LEIDEN_EINVAL;
  if (g.n > 0 && !it.membership_out) return LEIDEN_EINVAL;
  if (it.reserved != 0) return LEIDEN_EINVAL;
  if (it.mode == LEIDEN_STATIC) return LEIDEN_OK;
  if (it.mode != LEIDEN_ND && it.mode != LEIDEN_DS && it.mode != LEIDEN_DF) return LEIDEN_EINVAL;
  if (g.n > 0 && !it.prior) return LEIDEN_EINVAL;
  if (it.del.count < 0 || it.ins.count < 0) return LEIDEN_EINVAL;
  if (it.del.count > 0 && (!it.del.src || !it.del.dst || !it.del.w)) return LEIDEN_EINVAL;
  if (it.ins.count > 0 && (!it.ins.src || !it.ins.dst || !it.ins.w)) return LEIDEN_EINVAL;
  return LEIDEN_OK;
}

// (Re)captures upload + kernel + download into a CUDA graph for opts `so`.
int capture(leiden_batch *b, const SmallOpts &so) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->have_exec = false;
  const size_t smem = small_dyn_smem(b->threads);
  if (cudaFuncSetAttribute((const void *)small_leiden_k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return LEIDEN_ECUDA;
  }
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return LEIDEN_ECUDA;
  }
  SmallHeader *hdr = reinterpret_cast<SmallHeader *>(b->d_desc);
  const SmallJob *jobs = reinterpret_cast<const SmallJob *>(b->d_desc + sizeof(SmallHeader));
  cudaMemcpyAsync(b->d_desc, b->h_desc, b->desc_bytes, cudaMemcpyHostToDevice, b->cap);
  small_leiden_k<<<(unsigned)(b->sms * b->bps), b->threads, smem, b->cap>>>(hdr, jobs, so, b->d_res);
  cudaMemcpyAsync(b->h_res, b->d_res, b->res_bytes, cudaMemcpyDeviceToHost, b->cap);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(b->cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return LEIDEN_ECUDA;
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return LEIDEN_ECUDA;
  }
  b->graph = g;
  b->captured = so;
  b->have_exec = true;
  return LEIDEN_OK;
}

bool same_opts(const SmallOpts &a, const SmallOpts &b) { return memcmp(&a, &b, sizeof(SmallOpts)) == 0; }

}  // namespace

extern "C" int leiden_batch_create(leiden_batch **out, void *stream, int32_t max_graphs, int64_t max_total_n,
                                   int64_t max_total_nnz, int32_t threads, int32_t blocks_per_sm) {
  if (!out || max_graphs < 1 || max_total_n < 0 || max_total_nnz < 0) return LEIDEN_EINVAL;
  // measured on 64 planted-partition graphs of 10^4 vertices: 512 threads and
  // one block per SM 87 ms, 256 x 2 150 ms, 128 x 4 268 ms
  if (threads == 0) threads = 512;
  if (blocks_per_sm == 0) blocks_per_sm = 1;
  if (threads < 128 || threads > 512 || threads % 32) return LEIDEN_EINVAL;
  if (blocks_per_sm < 1 || blocks_per_sm > 4) return LEIDEN_EINVAL;
  leiden_batch *b = new leiden_batch();
  b->st = (cudaStream_t)stream;
  b->threads = threads;
  b->bps = blocks_per_sm;
  b->max_graphs = max_graphs;
  b->max_n = max_total_n;
  b->max_nnz = max_total_nnz;
  int rc = LEIDEN_OK;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    rc = LEIDEN_ECUDA;
  }
  b->arena_bytes = small_layout_bound(max_total_n, max_total_nnz, max_graphs);
  b->desc_bytes = sizeof(SmallHeader) + (size_t)max_graphs * sizeof(SmallJob);
  b->res_bytes = (size_t)max_graphs * sizeof(SmallResult);
  if (!rc && (cudaMalloc(&b->arena, (size_t)b->arena_bytes) != cudaSuccess ||
              cudaMalloc(&b->d_desc, b->desc_bytes) != cudaSuccess ||
              cudaMalloc((void **)&b->d_res, b->res_bytes) != cudaSuccess ||
              cudaMallocHost(&b->h_desc, b->desc_bytes) != cudaSuccess ||
              cudaMallocHost((void **)&b->h_res, b->res_bytes) != cudaSuccess))
    rc = LEIDEN_ENOMEM;
  if (rc) {
    cudaGetLastError();
    release(b);
    delete b;
    return rc;
  }
  memset(b->h_desc, 0, b->desc_bytes);
  *out = b;
  return LEIDEN_OK;
}

extern "C" void leiden_batch_destroy(leiden_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  cudaStreamSynchronize(b->cap);
  release(b);
  delete b;
}

extern "C" int leiden_batch_device_bytes(leiden_batch *b, int64_t *out) {
  if (!b || !out) return LEIDEN_EINVAL;
  *out = b->arena_bytes + (int64_t)b->desc_bytes + (int64_t)b->res_bytes;
  return LEIDEN_OK;
}

extern "C" int leiden_batch_run(leiden_batch *b, int32_t count, const leiden_batch_item *items,
                                const leiden_opts *opts, leiden_batch_result *results) {
  if (!b || count < 0 || (count > 0 && (!items || !results))) return LEIDEN_EINVAL;
  if (count > b->max_graphs) return LEIDEN_ENOMEM;
  SmallOpts so{};
  int rc = opts_to_small(opts, &so);
  if (rc) return rc;
  int64_t sum_n = 0, sum_nnz = 0;
  for (int k = 0; k < count; k++) {
    rc = check_item(items[k]);
    if (rc) return rc;
    sum_n += items[k].g.n;
    sum_nnz += items[k].g.nnz;
  }
  if (sum_n > b->max_n || sum_nnz > b->max_nnz) return LEIDEN_ENOMEM;
  if (count == 0) return LEIDEN_OK;
  // largest graphs first, so the last graphs to start are the shortest
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return items[x].g.nnz + items[x].g.n > items[y].g.nnz + items[y].g.n;
  });
  SmallHeader *hdr = reinterpret_cast<SmallHeader *>(b->h_desc);
  SmallJob *jobs = reinterpret_cast<SmallJob *>(b->h_desc + sizeof(SmallHeader));
  memset(hdr, 0, sizeof(SmallHeader));
  hdr->count = count;
  hdr->next = 0;
  int64_t at = 0;
  for (int k = 0; k < count; k++) {
    const leiden_batch_item &it = items[order[k]];
    SmallJob &j = jobs[k];
    memset(&j, 0, sizeof(j));
    j.n = it.g.n;
    j.nnz = it.g.nnz;
    j.off = it.g.off;
    j.idx = it.g.idx;
    j.w = it.g.w;
    j.mode = it.mode;
    j.out = it.membership_out;
    j.result = order[k];
    if (it.mode != LEIDEN_STATIC) {
      j.prior = it.prior;
      j.nd = it.del.count;
      j.ni = it.ins.count;
      j.ds = it.del.src; j.dd = it.del.dst; j.dw = it.del.w;
      j.is = it.ins.src; j.id = it.ins.dst; j.iw = it.ins.w;
    }
    j.ws = b->arena + at;
    at += small_layout(it.g.n, it.g.nnz).total;
  }
  if (at > b->arena_bytes) return LEIDEN_ENOMEM;  // cannot happen within the totals; kept as a guard
  // the previous run's graph is still in flight until this stream point
  if (!b->have_exec || !same_opts(so, b->captured)) {
    cudaStreamSynchronize(b->st);
    rc = capture(b, so);
    if (rc) return rc;
  }
  note_launch();
  if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) {
    cudaGetLastError();
    return LEIDEN_ECUDA;
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return LEIDEN_ECUDA;
  for (int k = 0; k < count; k++) {
    const SmallResult &r = b->h_res[k];
    leiden_batch_result &o = results[k];
    memset(&o, 0, sizeof(o));
    o.status = r.status;
    o.passes = r.passes;
    o.affected0 = r.affected0;
    o.changed0 = r.changed0;
    const int np = std::min<int>(r.passes, LEIDEN_STATS_PASSES);
    for (int p = 0; p < np; p++) {
      o.iters[p] = r.iters[p];
      o.nv[p] = r.nv[p];
      o.nnz[p] = r.nnz[p];
      o.moves[p] = r.moves[p];
      o.refine_moves[p] = r.refine_moves[p];
    }
    if (r.status == LEIDEN_OK) {
      const i128 sq = (i128)(((unsigned __int128)r.sq_hi << 64) | (unsigned __int128)r.sq_lo);
      const i128 num = (i128)so.q * r.two_m * r.inside - (i128)so.p * sq;
      o.q = r.two_m == 0 ? 0.0 : (double)num / ((double)r.two_m * (double)r.two_m * (double)so.q);
    }
  }
  return LEIDEN_OK;
}
