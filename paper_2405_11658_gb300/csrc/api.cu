// api.cu -- C-ABI entry points and the host driver of the pass loop
// (Alg. leiden) for Static, ND, DS and DF Leiden on one GPU.
//
// The driver keeps every array of the current super-vertex graph resident in
// the context's workspace; it synchronises the stream once per local-moving
// iteration (to test the iteration's total delta-modularity against tau) and
// once per pass (to read the community count after renumbering).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.h"
#include "leiden.h"

using namespace lk;

namespace {
// NVTX range around a phase ("local_move", "refine", "aggregate"), so a
// profiler can select a phase's kernels; free when no tool is attached.
struct Phase {
  explicit Phase(const char *name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
};
}  // namespace

namespace lk {
static std::atomic<uint64_t> g_kernel_launches{0};
void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace lk

struct leiden_ctx {
  cudaStream_t st = nullptr;
  // a context restricted to some SMs owns a green context and its stream
  GreenCtx green{};
  bool owns_stream = false;
  int device = 0, sms = 152;
  int64_t max_n = 0, max_nnz = 0;
  TierTable tiers{};
  int agg_uniform = 0;   // aggregation policy (leiden_ctx_set_agg_policy)
  std::vector<void *> allocs;
  int64_t device_bytes = 0;
  // vertex arrays
  int32_t *Ctop, *Cp, *CB, *rep;
  int64_t *Kp, *Sp, *S2, *K0, *Ktmp;
  uint8_t *ch, *ch2, *processed, *affected, *stamp, *flag;
  int32_t *prop_i, *prop_c;
  i128 *prop_S;
  int32_t *vlist, *clist, *cv;
  int64_t *ccount, *coff, *ctdeg, *hoff, *cdist, *ccur, *off2tmp;
  int64_t *scanned, *koff_dev, *scan_tmp;
  int32_t *blockhist;
  // level graphs (ping-pong) and aggregation scratch
  int64_t *goff[2];
  int32_t *gidx[2];
  int64_t *gw[2];
  int32_t *hidx;
  int64_t *hw;
  int32_t *gkeys;
  u64 *gvals;
  int64_t gcap = 0;
  int32_t *big;
  u64 *bcnt;
  int64_t *bpos;
  int64_t bcap = 0;
  HubWork hub{};
  int64_t hub_items = 0;
  u64 *ctr;
  // pinned host
  u64 *h_ctr;
  int64_t *h_koff;
  // diagnostics of the last failure
  char err[256] = {0};
  // statistics
  leiden_run_stats stats{};
  int timing = 0;
  std::vector<cudaEvent_t> evs;
  // auxiliary streams: the independent tier kernels of one sub-sweep run on
  // them concurrently, forked from and joined back into the context stream
  static constexpr int NAUX = LK_AUX_STREAMS > 0 ? LK_AUX_STREAMS : 1;
  cudaStream_t aux[NAUX] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[NAUX] = {};
};

cudaStream_t lk::ctx_stream(leiden_ctx *c) { return c->st; }

lk::CtxScope::CtxScope(leiden_ctx *c) {
  if (c && c->green.cu) pushed = green_push(c->green);
}
lk::CtxScope::~CtxScope() {
  if (pushed) green_pop();
}

namespace {

constexpr int MAX_KEYS = 256 * MAX_TIERS;

int dalloc(leiden_ctx *c, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return LEIDEN_ENOMEM;
  }
  c->allocs.push_back(*p);
  c->device_bytes += (int64_t)bytes;
  return LEIDEN_OK;
}

template <typename T>
int dal(leiden_ctx *c, T **p, int64_t count) {
  return dalloc(c, reinterpret_cast<void **>(p), (size_t)count * sizeof(T));
}

void free_all(leiden_ctx *c) {
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_koff) cudaFreeHost(c->h_koff);
  for (auto e : c->evs) cudaEventDestroy(e);
  c->evs.clear();
  for (int k = 0; k < leiden_ctx::NAUX; k++) {
    if (c->aux[k]) cudaStreamDestroy(c->aux[k]);
    if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
    c->aux[k] = nullptr;
    c->ev_join[k] = nullptr;
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  c->ev_fork = nullptr;
  c->h_ctr = nullptr;
  c->h_koff = nullptr;
}

int sync(leiden_ctx *c) {
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return LEIDEN_ECUDA;
  }
  return LEIDEN_OK;
}

int check_cuda(leiden_ctx *c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return LEIDEN_ECUDA;
  }
  return LEIDEN_OK;
}

// Device-side consistency flags (a full hashtable, a bad label): an internal
// error, reported as LEIDEN_ECUDA with the flag bits in the detail string.
int check_dev_flags(leiden_ctx *c, u64 flags) {
  if (!flags) return LEIDEN_OK;
  snprintf(c->err, sizeof(c->err), "device consistency check failed (flags 0x%llx)", flags);
  return LEIDEN_ECUDA;
}

int gamma_ratio(double gamma, int64_t *p, int64_t *q) {
  const double scaled = gamma * 1048576.0;
  if (!(gamma > 0.0) || scaled > 9.0e15) return LEIDEN_EINVAL;
  int64_t pp = (int64_t)scaled;
  if ((double)pp != scaled) return LEIDEN_EINVAL;
  int64_t qq = 1048576, a = pp, b = qq;
  while (b) { int64_t t = a % b; a = b; b = t; }
  *p = pp / a;
  *q = qq / a;
  return LEIDEN_OK;
}

int check_opts(const leiden_opts *o, int64_t *p, int64_t *q, int *log2S) {
  if (!o) return LEIDEN_EINVAL;
  if (o->max_iters < 1 || o->max_passes < 1 || !(o->tol >= 0.0) || !(o->tol_drop > 0.0)) return LEIDEN_EINVAL;
  if (o->sched != LEIDEN_DET && o->sched != LEIDEN_ASYNC) return LEIDEN_EINVAL;
  const int S = o->det_subsets;
  if (S < 1 || S > 256 || (S & (S - 1))) return LEIDEN_EINVAL;
  int k = 0;
  while ((1 << k) < S) k++;
  *log2S = k;  // both schedules walk the colour classes in order
  return gamma_ratio(o->gamma, p, q);
}

int check_graph(leiden_ctx *c, const leiden_csr *g) {
  if (!g || g->n < 0 || g->nnz < 0 || g->n >= INT32_MAX) return LEIDEN_EINVAL;
  // off has n + 1 entries even for an empty graph (the checks read off[0])
  if (!g->off || (g->nnz > 0 && (!g->idx || !g->w))) return LEIDEN_EINVAL;
  if (g->n > c->max_n || g->nnz > c->max_nnz) return LEIDEN_ENOMEM;
  return LEIDEN_OK;
}

// Per-run state shared by the phases.
struct Run {
  leiden_ctx *c;
  const leiden_opts *o;
  int64_t p, q, two_m, A;
  int log2S;
  bool dynamic;
  const uint8_t *in_range0;  // DS affected range in pass 0
  int64_t N;                 // vertices of the input graph
};

double denom(const Run &r) {
  // sum(S) / (2 m^2 q), with 2 m^2 = (2m)^2 / 2
  return (double)r.two_m * (double)r.two_m * 0.5 * (double)r.q;
}

i128 read_i128(const u64 *h) { return (i128)(((unsigned __int128)h[1] << 64) | (unsigned __int128)h[0]); }

template <typename WT>
MoveArgs<WT> base_args(const Run &r, GraphView<WT> g) {
  leiden_ctx *c = r.c;
  MoveArgs<WT> a{};
  a.g = g;
  a.C = c->Cp;
  a.K = c->Kp;
  a.Sig = c->Sp;
  a.processed = c->processed;
  a.in_range = nullptr;
  a.CB = c->CB;
  a.changed = c->ch;
  a.stamp = c->stamp;
  a.dynamic = 0;
  a.prop_i = c->prop_i;
  a.prop_c = c->prop_c;
  a.prop_S = c->prop_S;
  a.prop_count = &c->ctr[CTR_PROPS];
  a.A = r.A;
  a.p = r.p;
  a.gkeys = c->gkeys;
  a.gvals = c->gvals;
  a.glog2H = 0;
  a.big = c->big;
  a.ctr = c->ctr;
  return a;
}

struct Buckets {
  int64_t koff[MAX_KEYS + 1];
  int nkeys;
  int64_t maxdeg;
  int64_t kmax;  // largest weighted degree K' of the level
};

// out[0] = largest row length, out[1] = largest K'[i] of the level.
__global__ void maxdeg_k(const int64_t *off, const int64_t *K, int64_t n, u64 *out) {
  u64 m = 0, mk = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const u64 d = (u64)(off[i + 1] - off[i]);
    if (d > m) m = d;
    const u64 k = (u64)K[i];
    if (k > mk) mk = k;
  }
  for (int o = 16; o; o >>= 1) {
    const u64 y = __shfl_xor_sync(FULL_MASK, m, o);
    if (y > m) m = y;
    const u64 z = __shfl_xor_sync(FULL_MASK, mk, o);
    if (z > mk) mk = z;
  }
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(&out[0], m);
    if (mk) atomicMax(&out[1], mk);
  }
}

__global__ void count_u8_k(const uint8_t *a, int64_t n, u64 *out) {
  u64 s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] != 0;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

int64_t count_flags(leiden_ctx *c, const uint8_t *a, int64_t n) {
  cudaMemsetAsync(&c->ctr[CTR_SCRATCH0], 0, sizeof(u64), c->st);
  if (n > 0) LK_COUNTED count_u8_k<<<c->sms * 4, 256, 0, c->st>>>(a, n, &c->ctr[CTR_SCRATCH0]);
  cudaMemcpyAsync(&c->h_ctr[CTR_SCRATCH0], &c->ctr[CTR_SCRATCH0], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  if (sync(c)) return -1;
  return (int64_t)c->h_ctr[CTR_SCRATCH0];
}

int build_buckets(const Run &r, const int64_t *off, int64_t n, Buckets &b) {
  leiden_ctx *c = r.c;
  b.nkeys = (1 << r.log2S) * c->tiers.ntiers;
  launch_buckets(off, n, r.log2S, c->tiers, c->vlist, c->blockhist, c->scanned, c->koff_dev, c->scan_tmp, c->st);
  cudaMemsetAsync(&c->ctr[CTR_SCRATCH0], 0, 2 * sizeof(u64), c->st);
  if (n > 0) LK_COUNTED maxdeg_k<<<c->sms * 4, 256, 0, c->st>>>(off, c->Kp, n, &c->ctr[CTR_SCRATCH0]);
  cudaMemcpyAsync(c->h_koff, c->koff_dev, (size_t)(b.nkeys + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_SCRATCH0], &c->ctr[CTR_SCRATCH0], 2 * sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  int rc = sync(c);
  if (rc) return rc;
  memcpy(b.koff, c->h_koff, (size_t)(b.nkeys + 1) * sizeof(int64_t));
  b.maxdeg = (int64_t)c->h_ctr[CTR_SCRATCH0];
  b.kmax = (int64_t)c->h_ctr[CTR_SCRATCH0 + 1];
  return LEIDEN_OK;
}

// Width of the decide kernels' candidate scores for one level.  A vertex i
// compares its candidates by A K_{i->c} - p K_i Sigma'_c (Eq. 2 scaled by
// 2m^2 q, without the terms common to all candidates); with K_{i->c} <= K_i
// and Sigma'_c <= 2m both products lie in [0, K_i 2m max(p, q)], so while
// Kmax 2m max(p, q) < 2^62 every score fits 64 bits, and while Kmax < 2^31
// every summed K_{i->c} fits the 32-bit table values.  Only levels with a
// super-vertex of a large share of 2m need 128 bits.  The move itself (the
// full Eq. 2 score, its sum over the iteration) is always 128-bit, so the
// width changes no decision.
bool narrow_scores(const Run &r, const Buckets &b) {
  const int64_t pq = r.p > r.q ? r.p : r.q;
  return b.kmax < ((int64_t)1 << 31) && (i128)b.kmax * r.two_m * pq < ((i128)1 << 62);
}

// Launch the decide kernels of every tier of colour class s.  DET: the tiers
// touch disjoint vertices and only read the shared state, so they run
// concurrently on the auxiliary streams.  ASYNC: the tiers run one after the
// other on the context stream, longest rows first, each seeing the moves the
// tiers before it committed -- on power-law graphs the high-degree vertices
// decide first, as they do in the paper's loop over vertex IDs.
template <typename WT, typename ST, bool REFINE, bool ASYNC>
void decide_class(const Run &r, MoveArgs<WT> a, const Buckets &b, int s) {
  leiden_ctx *c = r.c;
  const int nt = c->tiers.ntiers;
  int used = 0;
  const bool serial = ASYNC;
  const bool fork = LK_AUX_STREAMS > 0 && !serial;
  if (fork) cudaEventRecord(c->ev_fork, c->st);
  for (int tt = 1; tt < nt; tt++) {
    const int t = serial ? nt - tt : tt;
    const int key = s * nt + t;
    a.list = c->vlist + b.koff[key];
    a.list_n = b.koff[key + 1] - b.koff[key];
    if (a.list_n <= 0) continue;
    const int k = used % leiden_ctx::NAUX;
    cudaStream_t st = fork ? c->aux[k] : c->st;
    if (fork && used < leiden_ctx::NAUX) cudaStreamWaitEvent(st, c->ev_fork, 0);
    used++;
    const Tier &T = c->tiers.t[t];
    if (T.kind == TIER_GLOBAL) {
      // hub rows: multi-block path, in rounds whose tables fit the scratch
      // (a hub's table has at most 2 * nextpow2(min(maxdeg, |V'|)) slots)
      int64_t tmax = HUB_TABLE_MIN;
      while (tmax < 2 * std::min<int64_t>(b.maxdeg, a.g.n)) tmax <<= 1;
      const int64_t budget = LK_HUB_ROUND_SLOTS > 0
                                 ? std::min<int64_t>(c->gcap, std::max<int64_t>(LK_HUB_ROUND_SLOTS, tmax))
                                 : c->gcap;
      const int64_t per_round = std::max<int64_t>(1, std::min(budget / tmax, c->hub_items / (tmax / 4096)));
      const int32_t *list = a.list;
      const int64_t nl = a.list_n;
      for (int64_t k0 = 0; k0 < nl; k0 += per_round) {
        MoveArgs<WT> h = a;
        h.list = list + k0;
        h.list_n = std::min(per_round, nl - k0);
        launch_hubs<WT, ST, REFINE, ASYNC>(h, c->hub, c->sms, st);
      }
      continue;
    }
    launch_decide<WT, ST, REFINE, ASYNC>(T, a, c->sms, st);
  }
  for (int k = 0; fork && k < used && k < leiden_ctx::NAUX; k++) {
    cudaEventRecord(c->ev_join[k], c->aux[k]);
    cudaStreamWaitEvent(c->st, c->ev_join[k], 0);
  }
}

// Alg. leidenlm.  Returns l_i (or a negative error code).
template <typename WT, typename ST>
int local_move(Run &r, GraphView<WT> g, const Buckets &b, bool first_pass, double tau, int64_t *moves_out) {
  leiden_ctx *c = r.c;
  const bool async = r.o->sched == LEIDEN_ASYNC;
  const int nsub = 1 << r.log2S;
  MoveArgs<WT> a = base_args(r, g);
  a.in_range = first_pass ? r.in_range0 : nullptr;
  a.dynamic = (r.dynamic && first_pass) ? 1 : 0;
  const double den = denom(r);
  int li = 0;
  int64_t moves = 0;
  cudaMemsetAsync(&c->ctr[CTR_MOVES], 0, sizeof(u64), c->st);
  cudaMemsetAsync(&c->ctr[CTR_SCANNED_ENTRIES], 0, 3 * sizeof(u64), c->st);
  while (li < r.o->max_iters) {
    // every vertex is unprocessed in the first iteration of a pass, except in
    // the first pass of an update (its affected set only)
    a.spec = (li == 0 && !(r.dynamic && first_pass)) ? 1 : 0;
    cudaMemsetAsync(&c->ctr[CTR_SUMS_LO], 0, 2 * sizeof(u64), c->st);
    const bool long_rows = b.maxdeg > BIG_ROW;
    for (int s = 0; s < nsub; s++) {
      if (!async) cudaMemsetAsync(&c->ctr[CTR_PROPS], 0, sizeof(u64), c->st);
      if (long_rows) cudaMemsetAsync(&c->ctr[CTR_BIG], 0, sizeof(u64), c->st);
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (c->timing) {
        const size_t k = (size_t)c->stats.move_kernel_launches * 2;
        while (c->evs.size() < k + 2) {
          cudaEvent_t e;
          cudaEventCreate(&e);
          c->evs.push_back(e);
        }
        e0 = c->evs[k];
        e1 = c->evs[k + 1];
        cudaEventRecord(e0, c->st);
      }
      if (async) decide_class<WT, ST, false, true>(r, a, b, s);
      else decide_class<WT, ST, false, false>(r, a, b, s);
      if (c->timing) {
        cudaEventRecord(e1, c->st);
        c->stats.move_kernel_launches++;
      }
      if (!async)
        launch_apply_moves(c->prop_i, c->prop_c, c->prop_S, c->ctr, c->Cp, c->Kp, c->Sp, c->ch, c->processed,
                           g.off, g.idx, c->big, a.dynamic, c->sms, c->st);
      if (long_rows) launch_mark_big(c->big, &c->ctr[CTR_BIG], g.off, g.idx, c->processed, c->sms, c->st);
    }
    li++;
    cudaMemcpyAsync(c->h_ctr, c->ctr, CTR_COUNT * sizeof(u64), cudaMemcpyDeviceToHost, c->st);
    int rc = sync(c);
    if (rc) return rc;
    rc = check_dev_flags(c, c->h_ctr[CTR_ERROR]);
    if (rc) return rc;
    const i128 sumS = read_i128(&c->h_ctr[CTR_SUMS_LO]);
    if (r.two_m == 0 || (double)sumS / den <= tau) break;
  }
  moves = (int64_t)c->h_ctr[CTR_MOVES];
  *moves_out = moves;
  // algorithmic bytes of the decide kernels: per scanned entry idx + w + the
  // gathered C'[j]; per scanned vertex the list entry, the pruning flag (read
  // and write), off[i..i+1], C'[i], K'[i] and Sigma'[d]; per distinct
  // candidate community its Sigma'[c]
  const int64_t ent = (int64_t)c->h_ctr[CTR_SCANNED_ENTRIES];
  const int64_t ver = (int64_t)c->h_ctr[CTR_SCANNED_VERTICES];
  const int64_t cand = (int64_t)c->h_ctr[CTR_CANDIDATES];
  c->stats.move_scanned_entries += ent;
  c->stats.move_scanned_vertices += ver;
  const double bytes = (double)ent * (8.0 + sizeof(WT)) + (double)ver * 42.0 + (double)cand * 8.0;
  c->stats.move_bytes += bytes;
  if (first_pass) {
    c->stats.move0_bytes += bytes;
    c->stats.move0_scanned_entries += ent;
    c->stats.move0_kernel_launches = c->stats.move_kernel_launches;  // the first pass's launches come first
  }
  return li;
}

// Alg. leidenre: one sweep (DET: one sub-sweep per colour class).
template <typename WT, typename ST>
int refine(Run &r, GraphView<WT> g, const Buckets &b, bool all_changed, int64_t *moves_out) {
  leiden_ctx *c = r.c;
  const bool async = r.o->sched == LEIDEN_ASYNC;
  const int nsub = 1 << r.log2S;
  MoveArgs<WT> a = base_args(r, g);
  a.spec = all_changed ? 1 : 0;  // every vertex starts isolated in a changed bound
  cudaMemsetAsync(&c->ctr[CTR_MOVES], 0, sizeof(u64), c->st);
  if (!async) cudaMemsetAsync(c->stamp, 0, (size_t)(g.n > 0 ? g.n : 1), c->st);
  for (int s = 0; s < nsub; s++) {
    if (async) {
      decide_class<WT, ST, true, true>(r, a, b, s);
    } else {
      cudaMemsetAsync(&c->ctr[CTR_PROPS], 0, sizeof(u64), c->st);
      // stamps 1..255 name the sub-sweep a vertex proposed in; a stamp only
      // matters inside its own sub-sweep, so the array is cleared on wrap
      const uint8_t sv = (uint8_t)(s % 255 + 1);
      if (s > 0 && sv == 1) cudaMemsetAsync(c->stamp, 0, (size_t)(g.n > 0 ? g.n : 1), c->st);
      a.stamp_val = sv;
      decide_class<WT, ST, true, false>(r, a, b, s);
      launch_apply_refine(c->prop_i, c->prop_c, c->ctr, c->stamp, sv, c->Cp, c->Kp, c->Sp, c->sms, c->st);
    }
  }
  if (async) launch_clear_left(c->Sp, g.n, c->st);
  cudaMemcpyAsync(c->h_ctr, c->ctr, CTR_COUNT * sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  int rc = sync(c);
  if (rc) return rc;
  rc = check_dev_flags(c, c->h_ctr[CTR_ERROR]);
  if (rc) return rc;
  *moves_out = (int64_t)c->h_ctr[CTR_MOVES];
  return LEIDEN_OK;
}

AggWork agg_work(leiden_ctx *c) {
  AggWork w{};
  w.ccount = c->ccount; w.coff = c->coff; w.ctdeg = c->ctdeg; w.hoff = c->hoff; w.cdist = c->cdist;
  w.off2tmp = c->off2tmp; w.ccur = c->ccur; w.cv = c->cv; w.clist = c->clist;
  w.hidx = c->hidx; w.hw = c->hw; w.gkeys = c->gkeys; w.gvals = c->gvals; w.gcap = c->gcap;
  w.blockhist = c->blockhist; w.scanned = c->scanned; w.koff_dev = c->koff_dev; w.scan_tmp = c->scan_tmp;
  w.h_koff = c->h_koff; w.Kout = c->Kp; w.ctr = c->ctr; w.sms = c->sms;
  w.bcnt = c->bcnt; w.bpos = c->bpos; w.bcap = c->bcap;
  w.uniform = c->agg_uniform;
  return w;
}

// One pass body for a level graph g; returns 1 to stop, 0 to continue with
// the aggregated graph written to level buffer `dst`, or a negative error.
double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

template <typename WT, typename ST>
int pass_body(Run &r, GraphView<WT> g, int lp, double tau, int dst, int64_t *nc_out, int64_t *nnz_out,
              const Buckets &b, std::chrono::steady_clock::time_point t_start);

template <typename WT>
int pass(Run &r, GraphView<WT> g, int lp, double tau, int dst, int64_t *nc_out, int64_t *nnz_out) {
  const auto t_start = std::chrono::steady_clock::now();
  Buckets b;
  int rc = build_buckets(r, g.off, g.n, b);
  if (rc) return rc;
  if (b.koff[b.nkeys] != g.n) return LEIDEN_ECUDA;
  if (!LK_FORCE_WIDE_SCORES && narrow_scores(r, b)) return pass_body<WT, int64_t>(r, g, lp, tau, dst, nc_out, nnz_out, b, t_start);
  if (lp < LEIDEN_STATS_PASSES) r.c->stats.wide_passes |= 1u << lp;
  return pass_body<WT, i128>(r, g, lp, tau, dst, nc_out, nnz_out, b, t_start);
}

template <typename WT, typename ST>
int pass_body(Run &r, GraphView<WT> g, int lp, double tau, int dst, int64_t *nc_out, int64_t *nnz_out,
              const Buckets &b, std::chrono::steady_clock::time_point t_start) {
  leiden_ctx *c = r.c;
  const int64_t nv = g.n;
  const bool rec = lp < LEIDEN_STATS_PASSES;
  int rc;
  if (b.maxdeg > 0) {
    int lh = 1;
    while (((int64_t)1 << lh) < 2 * b.maxdeg) lh++;
    if (((int64_t)1 << lh) > c->gcap) return LEIDEN_ENOMEM;
  }
  int64_t moves = 0, rmoves = 0;
  int li;
  {
    Phase ph(lp == 0 ? "local_move_pass0" : "local_move");
    li = local_move<WT, ST>(r, g, b, lp == 0, tau, &moves);
  }
  if (li < 0) return li;
  if (lp == 0) c->stats.changed0 = count_flags(c, c->ch, nv);
  if (rec) c->stats.t_move_ms[lp] = ms_since(t_start);
  const auto t_ref = std::chrono::steady_clock::now();
  // Alg. leidensr, then the bounds, the break and the refinement
  launch_subset_renumber(nv, c->Cp, c->Sp, c->S2, c->ch, c->ch2, c->rep, c->st);
  std::swap(c->Sp, c->S2);
  std::swap(c->ch, c->ch2);
  if (nv > 0) cudaMemcpyAsync(c->CB, c->Cp, (size_t)nv * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st);
  launch_break(nv, c->Cp, c->Kp, c->Sp, c->ch, c->st);
  {
    Phase ph("refine");
    rc = refine<WT, ST>(r, g, b, !(r.dynamic && lp == 0), &rmoves);
  }
  if (rc) return rc;
  if (rec) c->stats.t_refine_ms[lp] = ms_since(t_ref);
  const auto t_agg = std::chrono::steady_clock::now();
  if (lp < LEIDEN_STATS_PASSES) {
    c->stats.passes = lp + 1;
    c->stats.iters[lp] = li;
    c->stats.nv[lp] = nv;
    c->stats.moves[lp] = moves;
    c->stats.refine_moves[lp] = rmoves;
  }
  if (lp > 0 && li <= 1) {  // globally converged
    if (rec) c->stats.t_pass_ms[lp] = ms_since(t_start);
    return 1;
  }
  launch_renumber(nv, c->Cp, c->flag, c->scanned, c->scan_tmp, c->ctr, c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_NCOMM], &c->ctr[CTR_NCOMM], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  rc = sync(c);
  if (rc) return rc;
  const int64_t nc = (int64_t)c->h_ctr[CTR_NCOMM];
  *nc_out = nc;
  if (nc == nv) {  // aggregation would not shrink the graph
    if (rec) c->stats.t_pass_ms[lp] = ms_since(t_start);
    return 1;
  }
  launch_lookup(r.N, c->Ctop, c->Cp, c->st);
  int64_t nnz2 = 0;
  {
    Phase ph("aggregate");
    rc = aggregate<WT>(g, c->Cp, nc, c->goff[dst], c->gidx[dst], c->gw[dst], &nnz2, agg_work(c), c->st);
  }
  if (rc) return rc;
  cudaMemcpyAsync(&c->h_ctr[CTR_ERROR], &c->ctr[CTR_ERROR], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  rc = sync(c);
  if (rc) return rc;
  rc = check_dev_flags(c, c->h_ctr[CTR_ERROR]);
  if (rc) return rc;
  *nnz_out = nnz2;
  if (rec) {
    c->stats.t_agg_ms[lp] = ms_since(t_agg);
    c->stats.t_pass_ms[lp] = ms_since(t_start);
  }
  return 0;
}

int run_leiden(Run &r, const leiden_csr *g0) {
  // the first pass uses the input graph directly (int32 weights), later
  // passes the workspace (int64); each pass picks its score width
  leiden_ctx *c = r.c;
  const int64_t N = g0->n;
  launch_iota(c->Ctop, N, c->st);
  double tau = r.o->tol;
  GraphView<int32_t> g32{N, g0->off, g0->idx, g0->w};
  GraphView<int64_t> g64{};
  int cur = -1;  // -1: level 0 (input graph); else level buffer index
  int64_t nv = N;
  int lp;
  int64_t nnz_cur = g0->nnz;
  for (lp = 0; lp < r.o->max_passes; lp++) {
    if (lp < LEIDEN_STATS_PASSES) c->stats.nnz[lp] = nnz_cur;
    const int dst = cur < 0 ? 0 : 1 - cur;
    int64_t nc = 0, nnz2 = 0;
    int rc = cur < 0 ? pass<int32_t>(r, g32, lp, tau, dst, &nc, &nnz2)
                     : pass<int64_t>(r, g64, lp, tau, dst, &nc, &nnz2);
    if (rc < 0) return rc;
    if (rc == 1) break;
    // next level: K' = Sigma' = row sums (written by the aggregation), C' =
    // identity, everything unprocessed, every community changed
    cur = dst;
    g64 = GraphView<int64_t>{nc, c->goff[cur], c->gidx[cur], c->gw[cur]};
    nv = nc;
    nnz_cur = nnz2;
    launch_copy_i64(c->Sp, c->Kp, nv, c->st);
    launch_iota(c->Cp, nv, c->st);
    cudaMemsetAsync(c->processed, 0, (size_t)(nv > 0 ? nv : 1), c->st);
    cudaMemsetAsync(c->ch, 1, (size_t)(nv > 0 ? nv : 1), c->st);
    tau /= r.o->tol_drop;
  }
  launch_lookup(N, c->Ctop, c->Cp, c->st);
  return check_cuda(c);
}

// Device-side validation of a caller's CSR (off, idx, w); LEIDEN_EINVAL on a
// malformed graph.  One read of the graph, so the kernels after it can index
// by the graph's own IDs without further checks.
int validate_graph(leiden_ctx *c, const leiden_csr *g) {
  cudaMemsetAsync(&c->ctr[CTR_ERROR], 0, sizeof(u64), c->st);
  launch_check_graph(g->n, g->nnz, g->off, g->idx, g->w, &c->ctr[CTR_ERROR], c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_ERROR], &c->ctr[CTR_ERROR], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  int rc = sync(c);
  if (rc) return rc;
  if (c->h_ctr[CTR_ERROR]) {
    snprintf(c->err, sizeof(c->err), "malformed CSR (flags 0x%llx)", c->h_ctr[CTR_ERROR]);
    cudaMemsetAsync(&c->ctr[CTR_ERROR], 0, sizeof(u64), c->st);
    return LEIDEN_EINVAL;
  }
  return LEIDEN_OK;
}

int setup_run(leiden_ctx *c, const leiden_csr *g, const leiden_opts *o, Run &r) {
  r.c = c;
  r.o = o;
  c->err[0] = 0;
  int rc = check_opts(o, &r.p, &r.q, &r.log2S);
  if (rc) return rc;
  rc = check_graph(c, g);
  if (rc) return rc;
  rc = validate_graph(c, g);
  if (rc) return rc;
  r.N = g->n;
  return LEIDEN_OK;
}

int finish_two_m(leiden_ctx *c, Run &r, const leiden_csr *g) {
  // 2m = total CSR weight of G^t, from its row sums (K0)
  cudaMemsetAsync(&c->ctr[CTR_SCRATCH0], 0, sizeof(u64), c->st);
  launch_sum_i64(c->K0, g->n, &c->ctr[CTR_SCRATCH0], c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_SCRATCH0], &c->ctr[CTR_SCRATCH0], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  int rc = sync(c);
  if (rc) return rc;
  r.two_m = (int64_t)c->h_ctr[CTR_SCRATCH0];
  if (r.two_m < 0 || r.two_m >= ((int64_t)1 << 40)) return LEIDEN_EOVERFLOW;
  r.A = r.two_m * r.q;
  return LEIDEN_OK;
}

// The u64 accumulators of Eq. 1 cannot wrap while nnz <= 2^32 (each weight is
// below 2^31), and the 128-bit numerator q 2m inside - p sum Sigma^2 stays exact
// while 2m < 2^40 (the bound every run checks).
constexpr int64_t kModMaxNnz = (int64_t)1 << 32;

int modularity_of(leiden_ctx *c, const leiden_csr *g, const int32_t *C, int64_t p, int64_t q, double *q_out) {
  if (g->nnz > kModMaxNnz) return LEIDEN_EOVERFLOW;
  GraphView<int32_t> gv{g->n, g->off, g->idx, g->w};
  launch_modularity_terms(gv, g->nnz, C, c->Ktmp, &c->ctr[CTR_SCRATCH0], &c->ctr[CTR_ERROR], c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_SCRATCH0], &c->ctr[CTR_SCRATCH0], 4 * sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_ERROR], &c->ctr[CTR_ERROR], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  int rc = sync(c);
  if (rc) return rc;
  if (c->h_ctr[CTR_ERROR]) {
    // the callers validated the graph and the labels first, so this is an
    // internal inconsistency; the kernels skipped every bad index
    cudaMemsetAsync(&c->ctr[CTR_ERROR], 0, sizeof(u64), c->st);
    return check_dev_flags(c, c->h_ctr[CTR_ERROR]);
  }
  const int64_t inside = (int64_t)c->h_ctr[CTR_SCRATCH0];
  const i128 sq = read_i128(&c->h_ctr[CTR_SCRATCH0 + 1]);
  const int64_t two_m = (int64_t)c->h_ctr[CTR_SCRATCH0 + 3];
  if (two_m < 0 || two_m >= ((int64_t)1 << 40)) return LEIDEN_EOVERFLOW;
  const i128 num = (i128)q * two_m * inside - (i128)p * sq;
  *q_out = two_m == 0 ? 0.0 : (double)num / ((double)two_m * (double)two_m * (double)q);
  return LEIDEN_OK;
}

void reset_stats(leiden_ctx *c) {
  c->stats = leiden_run_stats{};
}

// A run that stopped half-way may leave scratch tables or counters dirty;
// restore the context's invariants so the next call starts clean.
int fail_run(leiden_ctx *c, int rc) {
  cudaMemsetAsync(c->gkeys, 0xff, (size_t)c->gcap * sizeof(int32_t), c->st);
  cudaMemsetAsync(c->gvals, 0, (size_t)c->gcap * sizeof(u64), c->st);
  cudaMemsetAsync(c->ctr, 0, CTR_COUNT * sizeof(u64), c->st);
  cudaStreamSynchronize(c->st);
  return rc;
}

void finish_timing(leiden_ctx *c) {
  if (!c->timing) return;
  double ms = 0, ms0 = 0;
  for (int64_t k = 0; k < c->stats.move_kernel_launches; k++) {
    float t = 0;
    cudaEventElapsedTime(&t, c->evs[2 * k], c->evs[2 * k + 1]);
    ms += t;
    if (k < c->stats.move0_kernel_launches) ms0 += t;
  }
  c->stats.move_kernel_ms = ms;
  c->stats.move0_kernel_ms = ms0;
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

void leiden_opts_default(leiden_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->gamma = 1.0;
  o->tol = 0.01;
  o->tol_drop = 10.0;
  o->max_iters = 20;
  o->max_passes = 10;
  o->sched = LEIDEN_DET;
  o->det_subsets = 8;
  o->refine_all_first_pass = 0;
}

int leiden_ctx_set_tiers(leiden_ctx *c, const leiden_tier_table *t) {
  if (!c) return LEIDEN_EINVAL;
  if (!t) { c->tiers = default_tiers(); return LEIDEN_OK; }
  TierTable tt;
  if (tiers_from_public(t, &tt) != LEIDEN_OK) return LEIDEN_EINVAL;
  c->tiers = tt;
  return LEIDEN_OK;
}

int leiden_ctx_set_agg_policy(leiden_ctx *c, int32_t policy) {
  if (!c || (policy != LEIDEN_AGG_TIERED && policy != LEIDEN_AGG_UNIFORM)) return LEIDEN_EINVAL;
  c->agg_uniform = policy == LEIDEN_AGG_UNIFORM;
  return LEIDEN_OK;
}

int leiden_ctx_get_tiers(leiden_ctx *c, leiden_tier_table *out) {
  if (!c || !out) return LEIDEN_EINVAL;
  tiers_to_public(c->tiers, out);
  return LEIDEN_OK;
}

int leiden_ctx_device_bytes(leiden_ctx *c, int64_t *out) {
  if (!c || !out) return LEIDEN_EINVAL;
  *out = c->device_bytes;
  return LEIDEN_OK;
}

uint64_t leiden_kernel_launches(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

const char *leiden_strerror(int code) {
  switch (code) {
    case LEIDEN_OK: return "ok";
    case LEIDEN_EINVAL: return "invalid argument";
    case LEIDEN_ENOMEM: return "exceeds capacity or out of memory";
    case LEIDEN_EOVERFLOW: return "total edge weight too large (2m >= 2^40)";
    case LEIDEN_ETIMEOUT: return "bounded device wait expired";
    case LEIDEN_ECUDA: return "CUDA error";
    default: return "unknown error";
  }
}

}  // extern "C"

namespace {
// Allocates the workspace of a context whose stream, device and SM count are
// set; on failure frees what it allocated (the caller deletes c).
int ctx_init(leiden_ctx *c, int64_t max_n, int64_t max_nnz) {
  c->max_n = max_n;
  c->max_nnz = max_nnz;
  c->tiers = default_tiers();
  const int64_t n1 = max_n + 1, m = max_nnz > 0 ? max_nnz : 1;
  const int64_t bh = bucket_blockhist_elems(max_n, MAX_KEYS);
  const int64_t scan_n = std::max<int64_t>(bh, 6 * n1 + 8);
  c->gcap = std::max<int64_t>(m, (int64_t)1 << 22);
  int rc = LEIDEN_OK;
  rc |= dal(c, &c->Ctop, n1); rc |= dal(c, &c->Cp, n1); rc |= dal(c, &c->CB, n1); rc |= dal(c, &c->rep, n1);
  rc |= dal(c, &c->Kp, n1); rc |= dal(c, &c->Sp, n1); rc |= dal(c, &c->S2, n1); rc |= dal(c, &c->K0, n1);
  rc |= dal(c, &c->Ktmp, n1);
  rc |= dal(c, &c->ch, n1 + 16); rc |= dal(c, &c->ch2, n1 + 16); rc |= dal(c, &c->processed, n1 + 16);
  rc |= dal(c, &c->affected, n1 + 16); rc |= dal(c, &c->stamp, n1 + 16); rc |= dal(c, &c->flag, n1 + 16);
  rc |= dal(c, &c->prop_i, n1); rc |= dal(c, &c->prop_c, n1); rc |= dal(c, &c->prop_S, n1);
  rc |= dal(c, &c->vlist, n1); rc |= dal(c, &c->clist, n1); rc |= dal(c, &c->cv, n1);
  rc |= dal(c, &c->ccount, n1); rc |= dal(c, &c->coff, n1); rc |= dal(c, &c->ctdeg, n1);
  rc |= dal(c, &c->hoff, n1); rc |= dal(c, &c->cdist, n1); rc |= dal(c, &c->ccur, n1);
  rc |= dal(c, &c->off2tmp, 6 * n1 + 8);
  rc |= dal(c, &c->scanned, scan_n + 1); rc |= dal(c, &c->koff_dev, MAX_KEYS + 1);
  rc |= dal(c, &c->scan_tmp, scan_tmp_elems(scan_n) + 1);
  rc |= dal(c, &c->blockhist, bh);
  for (int k = 0; k < 2; k++) {
    rc |= dal(c, &c->goff[k], n1); rc |= dal(c, &c->gidx[k], m); rc |= dal(c, &c->gw[k], m);
  }
  rc |= dal(c, &c->hidx, m); rc |= dal(c, &c->hw, m);
  rc |= dal(c, &c->gkeys, c->gcap); rc |= dal(c, &c->gvals, c->gcap);
  rc |= dal(c, &c->ctr, CTR_COUNT);
  rc |= dal(c, &c->big, n1);
  // giant-community buckets: a community of total degree T > 2048 gets at most
  // 2 * ceil(T / 2048) <= T / 512 buckets, so the total stays below nnz / 512
  c->bcap = m / 256 + n1 + 16;
  rc |= dal(c, &c->bcnt, c->bcap); rc |= dal(c, &c->bpos, c->bcap);
  rc |= dal(c, &c->hub.tsz, n1); rc |= dal(c, &c->hub.toff, n1);
  rc |= dal(c, &c->hub.ioff, n1); rc |= dal(c, &c->hub.soff, n1);
  rc |= dal(c, &c->hub.tot, 4);
  c->hub_items = c->gcap / 4096 + 1024;
  rc |= dal(c, &c->hub.psc, c->hub_items); rc |= dal(c, &c->hub.pc, c->hub_items);
  rc |= dal(c, &c->hub.pkid, c->hub_items);
  if (rc == LEIDEN_OK) {
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) rc = LEIDEN_ENOMEM;
    for (int k = 0; k < leiden_ctx::NAUX && rc == LEIDEN_OK; k++) {
      if (cudaStreamCreateWithFlags(&c->aux[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming) != cudaSuccess)
        rc = LEIDEN_ENOMEM;
    }
  }
  if (rc == LEIDEN_OK) {
    if (cudaMallocHost((void **)&c->h_ctr, CTR_COUNT * sizeof(u64)) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_koff, (MAX_KEYS + 8) * sizeof(int64_t)) != cudaSuccess)
      rc = LEIDEN_ENOMEM;
  }
  if (rc != LEIDEN_OK) {
    cudaGetLastError();
    free_all(c);
    return LEIDEN_ENOMEM;
  }
  cudaMemsetAsync(c->ctr, 0, CTR_COUNT * sizeof(u64), c->st);
  // the global scratch tables start (and are always left) empty
  cudaMemsetAsync(c->gkeys, 0xff, (size_t)c->gcap * sizeof(int32_t), c->st);
  cudaMemsetAsync(c->gvals, 0, (size_t)c->gcap * sizeof(u64), c->st);
  if (sync(c)) { free_all(c); return LEIDEN_ECUDA; }
  return LEIDEN_OK;
}
}  // namespace

extern "C" {

int leiden_ctx_create(leiden_ctx **out, void *cuda_stream, int64_t max_n, int64_t max_nnz) {
  if (!out || max_n < 0 || max_nnz < 0 || max_n >= INT32_MAX) return LEIDEN_EINVAL;
  *out = nullptr;
  leiden_ctx *c = new leiden_ctx();
  c->st = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return LEIDEN_ECUDA; }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  const int rc = ctx_init(c, max_n, max_nnz);
  if (rc) { delete c; return rc; }
  *out = c;
  return LEIDEN_OK;
}

int leiden_ctx_create_sm(leiden_ctx **out, int32_t sm_count, int64_t max_n, int64_t max_nnz,
                         int32_t *sms_granted) {
  if (!out || sm_count < 1 || max_n < 0 || max_nnz < 0 || max_n >= INT32_MAX) return LEIDEN_EINVAL;
  *out = nullptr;
  leiden_ctx *c = new leiden_ctx();
  if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return LEIDEN_ECUDA; }
  int rc = green_create(c->device, sm_count, &c->green);
  if (rc) { delete c; return rc; }
  c->sms = c->green.sms;
  rc = LEIDEN_ECUDA;
  if (green_push(c->green)) {
    // the context stream and the auxiliary streams are created while the
    // green context is current, so every kernel runs on its SMs
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) == cudaSuccess) {
      c->owns_stream = true;
      rc = ctx_init(c, max_n, max_nnz);
      if (rc) cudaStreamDestroy(c->st);
    } else {
      cudaGetLastError();
    }
    green_pop();
  }
  if (rc) {
    green_destroy(&c->green);
    delete c;
    return rc;
  }
  if (sms_granted) *sms_granted = c->sms;
  *out = c;
  return LEIDEN_OK;
}

int leiden_ctx_sm_count(leiden_ctx *c, int32_t *out) {
  if (!c || !out) return LEIDEN_EINVAL;
  *out = c->sms;
  return LEIDEN_OK;
}


void leiden_ctx_destroy(leiden_ctx *c) {
  if (!c) return;
  {
    CtxScope scope(c);
    cudaStreamSynchronize(c->st);
    free_all(c);
    if (c->owns_stream) cudaStreamDestroy(c->st);
  }
  if (c->green.green) green_destroy(&c->green);
  delete c;
}

int leiden_ctx_set_timing(leiden_ctx *c, int32_t enable) {
  if (!c) return LEIDEN_EINVAL;
  c->timing = enable ? 1 : 0;
  return LEIDEN_OK;
}

const char *leiden_ctx_last_error(leiden_ctx *c) {
  if (!c) return "no context";
  return c->err;
}

int leiden_get_stats(leiden_ctx *c, leiden_run_stats *out) {
  if (!c || !out) return LEIDEN_EINVAL;
  *out = c->stats;
  return LEIDEN_OK;
}

int leiden_static(leiden_ctx *c, const leiden_csr *g, const leiden_opts *o, int32_t *membership_out,
                  double *q_out) {
  if (!c || (!membership_out && g && g->n > 0)) return LEIDEN_EINVAL;
  CtxScope scope(c);
  const auto t0 = std::chrono::steady_clock::now();
  Run r{};
  int rc = setup_run(c, g, o, r);
  if (rc) return rc;
  reset_stats(c);
  const int64_t n = g->n;
  GraphView<int32_t> gv{n, g->off, g->idx, g->w};
  launch_row_sums(gv, c->K0, c->st);
  rc = finish_two_m(c, r, g);
  if (rc) return rc;
  // Static: C' = identity, K' = K, Sigma' = K, every community changed,
  // every vertex affected and in range
  launch_copy_i64(c->Kp, c->K0, n, c->st);
  launch_copy_i64(c->Sp, c->K0, n, c->st);
  launch_iota(c->Cp, n, c->st);
  cudaMemsetAsync(c->ch, 1, (size_t)(n > 0 ? n : 1), c->st);
  cudaMemsetAsync(c->processed, 0, (size_t)(n > 0 ? n : 1), c->st);
  r.dynamic = false;
  r.in_range0 = nullptr;
  c->stats.affected0 = n;
  rc = run_leiden(r, g);
  if (rc) return fail_run(c, rc);
  launch_canonical(n, c->Ctop, membership_out, c->rep, c->flag, c->scanned, c->scan_tmp, c->st);
  rc = sync(c);
  if (rc) return rc;
  if (q_out) {
    rc = modularity_of(c, g, membership_out, r.p, r.q, q_out);
    if (rc) return rc;
  }
  finish_timing(c);
  c->stats.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return LEIDEN_OK;
}

int leiden_update(leiden_ctx *c, const leiden_csr *g, const int32_t *prior_membership, const int64_t *prior_K,
                  const int64_t *prior_Sigma, const leiden_edges *del, const leiden_edges *ins, int32_t mode,
                  const leiden_opts *o, int32_t *membership_out, int64_t *K_out, int64_t *Sigma_out,
                  double *q_out) {
  if (!c) return LEIDEN_EINVAL;
  CtxScope scope(c);
  const auto t0 = std::chrono::steady_clock::now();
  Run r{};
  int rc = setup_run(c, g, o, r);
  if (rc) return rc;
  if (mode != LEIDEN_ND && mode != LEIDEN_DS && mode != LEIDEN_DF) return LEIDEN_EINVAL;
  const int64_t n = g->n;
  if (n > 0 && (!prior_membership || !membership_out)) return LEIDEN_EINVAL;
  if ((prior_K == nullptr) != (prior_Sigma == nullptr)) return LEIDEN_EINVAL;
  const int64_t nd = del ? del->count : 0, ni = ins ? ins->count : 0;
  if (nd < 0 || ni < 0) return LEIDEN_EINVAL;
  if ((nd > 0 && (!del->src || !del->dst || !del->w)) || (ni > 0 && (!ins->src || !ins->dst || !ins->w)))
    return LEIDEN_EINVAL;
  if (2 * ni > c->max_nnz || 2 * nd > c->max_nnz) return LEIDEN_ENOMEM;
  reset_stats(c);
  // batch IDs must lie in [0, n), no self-loops, positive weights
  cudaMemsetAsync(&c->ctr[CTR_ERROR], 0, sizeof(u64), c->st);
  if (nd) launch_check_ids(nd, del->src, del->dst, del->w, n, &c->ctr[CTR_ERROR], c->st);
  if (ni) launch_check_ids(ni, ins->src, ins->dst, ins->w, n, &c->ctr[CTR_ERROR], c->st);
  launch_check_range(prior_membership, n, n, &c->ctr[CTR_ERROR], c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_ERROR], &c->ctr[CTR_ERROR], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  rc = sync(c);
  if (rc) return rc;
  if (c->h_ctr[CTR_ERROR]) {
    snprintf(c->err, sizeof(c->err), "batch IDs or prior labels out of range (flags 0x%llx)",
             c->h_ctr[CTR_ERROR]);
    cudaMemsetAsync(&c->ctr[CTR_ERROR], 0, sizeof(u64), c->st);
    return LEIDEN_EINVAL;
  }

  GraphView<int32_t> gv{n, g->off, g->idx, g->w};
  launch_row_sums(gv, c->K0, c->st);  // K^t of G^t, also the source of 2m
  rc = finish_two_m(c, r, g);
  if (rc) return rc;
  // Alg. update: K^t, Sigma^t from the auxiliary information, or recomputed
  if (prior_K) {
    launch_copy_i64(c->Kp, prior_K, n, c->st);
    launch_copy_i64(c->Sp, prior_Sigma, n, c->st);
    if (nd) launch_update_weights(nd, del->src, del->dst, del->w, -1, prior_membership, c->Kp, c->Sp, c->st);
    if (ni) launch_update_weights(ni, ins->src, ins->dst, ins->w, +1, prior_membership, c->Kp, c->Sp, c->st);
    launch_copy_i64(c->K0, c->Kp, n, c->st);  // K^t as Alg. update gives it
  } else {
    launch_copy_i64(c->Kp, c->K0, n, c->st);
    launch_sigma_from(n, prior_membership, c->Kp, c->Sp, c->st);
  }
  // changedCommunities (Alg. leiden, dynamic branch)
  cudaMemsetAsync(c->ch, 0, (size_t)(n > 0 ? n : 1), c->st);
  if (!o->refine_all_first_pass) {
    if (nd) launch_changed_communities(nd, del->src, del->dst, prior_membership, c->ch, c->st);
    if (ni) launch_changed_communities(ni, ins->src, ins->dst, prior_membership, c->ch, c->st);
  } else {
    cudaMemsetAsync(c->ch, 1, (size_t)(n > 0 ? n : 1), c->st);
  }
  // affected vertices (Alg. naive / delta / frontier)
  r.in_range0 = nullptr;
  if (mode == LEIDEN_ND) {
    cudaMemsetAsync(c->processed, 0, (size_t)(n > 0 ? n : 1), c->st);
  } else {
    cudaMemsetAsync(c->affected, 0, (size_t)(n > 0 ? n : 1), c->st);
    if (mode == LEIDEN_DF) {
      if (nd) launch_mark_df(nd, del->src, del->dst, prior_membership, 1, c->affected, c->st);
      if (ni) launch_mark_df(ni, ins->src, ins->dst, prior_membership, 0, c->affected, c->st);
    } else {
      DsWork w{};
      w.cnt = c->ccount; w.soff = c->coff; w.cur = c->ccur;
      w.sdst = c->hidx; w.swt = reinterpret_cast<int32_t *>(c->hw);
      w.scan_tmp = c->scan_tmp; w.dE = c->flag; w.dC = c->stamp;
      launch_mark_ds(n, g->off, g->idx, prior_membership, c->Kp, c->Sp, r.A, r.p, nd, nd ? del->src : nullptr,
                     nd ? del->dst : nullptr, ni, ni ? ins->src : nullptr, ni ? ins->dst : nullptr,
                     ni ? ins->w : nullptr, c->affected, w, c->st);
      r.in_range0 = c->affected;
    }
    launch_invert_u8(c->processed, c->affected, n, c->st);
  }
  if (n > 0) cudaMemcpyAsync(c->Cp, prior_membership, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st);
  c->stats.affected0 = mode == LEIDEN_ND ? n : count_flags(c, c->affected, n);
  r.dynamic = true;
  rc = run_leiden(r, g);
  if (rc) return fail_run(c, rc);
  launch_canonical(n, c->Ctop, membership_out, c->rep, c->flag, c->scanned, c->scan_tmp, c->st);
  if (K_out) launch_copy_i64(K_out, c->K0, n, c->st);
  if (Sigma_out) launch_sigma_from(n, membership_out, c->K0, Sigma_out, c->st);
  rc = sync(c);
  if (rc) return rc;
  if (q_out) {
    rc = modularity_of(c, g, membership_out, r.p, r.q, q_out);
    if (rc) return rc;
  }
  finish_timing(c);
  c->stats.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return LEIDEN_OK;
}

int leiden_modularity(leiden_ctx *c, const leiden_csr *g, const int32_t *membership, double gamma, double *q_out) {
  if (!c || !q_out) return LEIDEN_EINVAL;
  CtxScope scope(c);
  int rc = check_graph(c, g);
  if (rc) return rc;
  if (g->n > 0 && !membership) return LEIDEN_EINVAL;
  rc = validate_graph(c, g);
  if (rc) return rc;
  cudaMemsetAsync(&c->ctr[CTR_ERROR], 0, sizeof(u64), c->st);
  launch_check_range(membership, g->n, g->n, &c->ctr[CTR_ERROR], c->st);
  cudaMemcpyAsync(&c->h_ctr[CTR_ERROR], &c->ctr[CTR_ERROR], sizeof(u64), cudaMemcpyDeviceToHost, c->st);
  rc = sync(c);
  if (rc) return rc;
  if (c->h_ctr[CTR_ERROR]) {
    cudaMemsetAsync(&c->ctr[CTR_ERROR], 0, sizeof(u64), c->st);
    return LEIDEN_EINVAL;
  }
  int64_t p, q;
  rc = gamma_ratio(gamma, &p, &q);
  if (rc) return rc;
  return modularity_of(c, g, membership, p, q, q_out);
}

int leiden_apply_batch(leiden_ctx *c, const leiden_csr *g, const leiden_edges *del, const leiden_edges *ins,
                       int64_t *off_out, int32_t *idx_out, int32_t *w_out, int64_t cap_nnz, int64_t *nnz_out) {
  if (!c || !off_out || !nnz_out || cap_nnz < 0) return LEIDEN_EINVAL;
  CtxScope scope(c);
  int rc = check_graph(c, g);
  if (rc) return rc;
  const int64_t nd = del ? del->count : 0, ni = ins ? ins->count : 0;
  if (nd < 0 || ni < 0) return LEIDEN_EINVAL;
  if ((nd > 0 && (!del->src || !del->dst || !del->w)) || (ni > 0 && (!ins->src || !ins->dst || !ins->w)))
    return LEIDEN_EINVAL;
  if (2 * (ni + nd) > c->max_nnz) return LEIDEN_ENOMEM;
  if (cap_nnz > 0 && (!idx_out || !w_out)) return LEIDEN_EINVAL;
  rc = validate_graph(c, g);
  if (rc) return rc;
  // scratch borrowed from the workspace (all free outside a Leiden run)
  const int64_t U = 2 * (ni + nd);
  BatchWork w{};
  w.cnt = c->ccount; w.uoff = c->coff; w.cur = c->ccur;
  w.ut = c->hidx;
  w.uw = reinterpret_cast<int32_t *>(c->hw);
  w.Rp = reinterpret_cast<int32_t *>(c->hw) + c->max_nnz;
  w.Np = c->gidx[0];
  uint8_t *scratch = reinterpret_cast<uint8_t *>(c->gvals);    // 8 * gcap >= U + nnz / 8 + 16 bytes
  w.uk = scratch;
  w.bits = reinterpret_cast<uint32_t *>(scratch + ((U + 15) & ~(int64_t)15));
  w.tflag = c->flag; w.tpos = c->cdist; w.trow = c->cv;
  w.newdeg = c->ctdeg;
  w.scan_tmp = c->scan_tmp;
  w.err = &c->ctr[CTR_ERROR];
  rc = apply_batch(g->n, g->off, g->idx, g->w, nd, nd ? del->src : nullptr, nd ? del->dst : nullptr,
                   nd ? del->w : nullptr, ni, ni ? ins->src : nullptr, ni ? ins->dst : nullptr,
                   ni ? ins->w : nullptr, off_out, idx_out, w_out, cap_nnz, nnz_out, w, c->st);
  // the record kinds and the row-start bits borrowed the scratch values:
  // leave them zero again
  const int64_t used = ((U + 15) & ~(int64_t)15) + ((g->nnz + 31) / 32 + 1) * 4;
  cudaMemsetAsync(c->gvals, 0, (size_t)used, c->st);
  const int rc2 = sync(c);
  return rc ? rc : rc2;
}

}  // extern "C"
