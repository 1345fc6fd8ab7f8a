// server.cu -- the serving loop (leiden_server_*): resident graphs admitted
// against a device-memory budget, per-graph FIFO queues of update batches,
// and worker threads that pick work as soon as a graph and a worker are free
// (continuous batching):
//   * `small_workers` small-graph workers, each draining every ready request
//     of a small graph into one persistent launch (leiden_batch_run) after
//     building each G^t, so one launch can start while another runs;
//   * `large_slots` workers, each with its own leiden_ctx and stream, run the
//     updates of large graphs concurrently on the device.
// Host code only; every step on the device is a library call.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "leiden.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  int64_t id = 0;
  int32_t graph = 0;
  bool is_static = false;
  std::vector<int32_t> ds, dd, dw, is, id_, iw;
  Clock::time_point t_submit, t_start;
  leiden_request_info info{};
  bool done = false;
};

struct Resident {
  int32_t id = 0;
  int64_t n = 0, nnz = 0, cap = 0;
  bool small = false;
  int64_t *off[2] = {};
  int32_t *idx[2] = {}, *w[2] = {};
  int32_t *C[2] = {};
  int64_t *K[2] = {}, *Sig[2] = {};
  int csr = 0, mem = 0;   // current CSR and membership buffers
  bool has_aux = false;   // K / Sigma of the current membership are valid
  bool tuned = false;     // `tiers` picked by the autotuner for this graph
  leiden_tier_table tiers{};
  bool busy = false;
  std::deque<Request *> queue;
  std::vector<void *> allocs;
  int64_t bytes = 0;
};

// Device staging of batch arrays, grown on demand.
struct Staging {
  int32_t *buf = nullptr;
  int64_t cap = 0;   // int32 elements
};

}  // namespace

struct leiden_server {
  leiden_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;     // work available / request done / graph idle
  bool stop = false;
  int64_t next_req = 1;
  int32_t next_graph = 1;
  std::unordered_map<int32_t, Resident *> graphs;
  std::unordered_map<int64_t, Request *> reqs;
  int64_t pending = 0;            // requests not yet done
  int64_t workspace_bytes = 0, resident_bytes = 0;
  leiden_server_stats st{};
  // workers
  std::vector<std::thread> threads;
  std::vector<leiden_ctx *> large_ctx;
  std::vector<cudaStream_t> large_st;
  std::vector<Staging> large_stage;
  struct Small {
    leiden_ctx *ctx = nullptr;
    leiden_batch *batch = nullptr;
    cudaStream_t st = nullptr;
    Staging stage;
  };
  std::vector<Small> small;
};

namespace {

int grow(leiden_server *s, Staging &sg, int64_t need) {
  if (need <= sg.cap) return LEIDEN_OK;
  int64_t cap = std::max<int64_t>(need, 2 * sg.cap);
  cap = std::max<int64_t>(cap, 1 << 16);
  int32_t *p = nullptr;
  if (cudaMalloc(&p, (size_t)cap * 4) != cudaSuccess) { cudaGetLastError(); return LEIDEN_ENOMEM; }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->workspace_bytes += (cap - sg.cap) * 4;
  }
  if (sg.buf) cudaFree(sg.buf);
  sg.buf = p;
  sg.cap = cap;
  return LEIDEN_OK;
}

// Copies a request's batch to device staging at `at`; fills del / ins.
void upload_batch(const Request &r, int32_t *at, cudaStream_t st, leiden_edges *del, leiden_edges *ins) {
  const int64_t nd = (int64_t)r.ds.size(), ni = (int64_t)r.is.size();
  int32_t *p = at;
  auto put = [&](const std::vector<int32_t> &v) {
    int32_t *q = p;
    if (!v.empty()) cudaMemcpyAsync(q, v.data(), v.size() * 4, cudaMemcpyHostToDevice, st);
    p += v.size();
    return q;
  };
  del->count = nd;
  del->src = put(r.ds); del->dst = put(r.dd); del->w = put(r.dw);
  ins->count = ni;
  ins->src = put(r.is); ins->dst = put(r.id_); ins->w = put(r.iw);
}

int64_t batch_words(const Request &r) { return 3 * (int64_t)(r.ds.size() + r.is.size()); }

leiden_csr csr_of(const Resident &g, int k, int64_t nnz) {
  leiden_csr c{};
  c.n = g.n;
  c.nnz = nnz;
  c.off = g.off[k];
  c.idx = g.idx[k];
  c.w = g.w[k];
  return c;
}

void finish(leiden_server *s, Resident *g, std::vector<Request *> &done) {
  const auto t = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  for (Request *r : done) {
    r->info.latency_ms = ms_between(r->t_submit, t);
    r->info.queue_ms = ms_between(r->t_submit, r->t_start);
    r->done = true;
    s->pending--;
    if (r->info.status == LEIDEN_OK) s->st.completed++; else s->st.failed++;
  }
  if (g) g->busy = false;
  s->cv.notify_all();
}

// One request of a large graph on worker k.
void run_large(leiden_server *s, int k, Resident *g, Request *r) {
  leiden_ctx *ctx = s->large_ctx[k];
  cudaStream_t st = s->large_st[k];
  leiden_request_info &info = r->info;
  info.graph = g->id;
  info.path = 1;
  int rc = LEIDEN_OK;
  double q = 0.0;
  leiden_ctx_set_tiers(ctx, g->tuned ? &g->tiers : nullptr);
  if (r->is_static) {
    leiden_csr c = csr_of(*g, g->csr, g->nnz);
    if (s->cfg.autotune_trials > 0) {
      rc = leiden_autotune(ctx, &c, &s->cfg.opts, s->cfg.autotune_trials, 1, &g->tiers, nullptr);
      g->tuned = rc == LEIDEN_OK;
    }
    if (!rc) rc = leiden_static(ctx, &c, &s->cfg.opts, g->C[g->mem], &q);
    if (!rc) g->has_aux = false;
  } else {
    rc = grow(s, s->large_stage[k], batch_words(*r));
    leiden_edges del{}, ins{};
    if (!rc) upload_batch(*r, s->large_stage[k].buf, st, &del, &ins);
    int64_t nnz2 = 0;
    const int nx = 1 - g->csr;
    leiden_csr cur = csr_of(*g, g->csr, g->nnz);
    if (!rc) rc = leiden_apply_batch(ctx, &cur, &del, &ins, g->off[nx], g->idx[nx], g->w[nx], g->cap, &nnz2);
    if (!rc) {
      leiden_csr nxt = csr_of(*g, nx, nnz2);
      const int mx = 1 - g->mem;
      rc = leiden_update(ctx, &nxt, g->C[g->mem], g->has_aux ? g->K[g->mem] : nullptr,
                         g->has_aux ? g->Sig[g->mem] : nullptr, &del, &ins, s->cfg.mode, &s->cfg.opts, g->C[mx],
                         g->K[mx], g->Sig[mx], &q);
      if (!rc) {
        g->csr = nx;
        g->nnz = nnz2;
        g->mem = mx;
        g->has_aux = true;
      }
    }
  }
  cudaStreamSynchronize(st);
  info.status = rc;
  info.q = q;
  info.n = g->n;
  info.nnz = g->nnz;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.large_runs++;
  }
  std::vector<Request *> d{r};
  finish(s, g, d);
}

// A small graph's request on the small worker's own context (all SMs on one
// graph): for the few-graph case, where one block per graph would be slower.
void run_small_alone(leiden_server *s, int w, Resident *g, Request *r) {
  leiden_server::Small &sw = s->small[w];
  leiden_request_info &info = r->info;
  info.graph = g->id;
  info.path = 2;
  int rc = LEIDEN_OK;
  double q = 0.0;
  const int mx = 1 - g->mem;
  if (r->is_static) {
    leiden_csr c = csr_of(*g, g->csr, g->nnz);
    rc = leiden_static(sw.ctx, &c, &s->cfg.opts, g->C[mx], &q);
    if (!rc) { g->mem = mx; g->has_aux = false; }
  } else {
    rc = grow(s, sw.stage, batch_words(*r));
    leiden_edges del{}, ins{};
    if (!rc) upload_batch(*r, sw.stage.buf, sw.st, &del, &ins);
    int64_t nnz2 = 0;
    const int nx = 1 - g->csr;
    leiden_csr cur = csr_of(*g, g->csr, g->nnz);
    if (!rc) rc = leiden_apply_batch(sw.ctx, &cur, &del, &ins, g->off[nx], g->idx[nx], g->w[nx], g->cap, &nnz2);
    if (!rc) {
      leiden_csr nxt = csr_of(*g, nx, nnz2);
      rc = leiden_update(sw.ctx, &nxt, g->C[g->mem], g->has_aux ? g->K[g->mem] : nullptr,
                         g->has_aux ? g->Sig[g->mem] : nullptr, &del, &ins, s->cfg.mode, &s->cfg.opts, g->C[mx],
                         g->K[mx], g->Sig[mx], &q);
      if (!rc) { g->csr = nx; g->nnz = nnz2; g->mem = mx; g->has_aux = true; }
    }
  }
  cudaStreamSynchronize(sw.st);
  info.status = rc;
  info.q = q;
  info.n = g->n;
  info.nnz = g->nnz;
  std::vector<Request *> d{r};
  finish(s, g, d);
}

// The ready requests of small graphs, in one persistent launch.
void run_small(leiden_server *s, int w, std::vector<std::pair<Resident *, Request *>> &work) {
  leiden_server::Small &sw = s->small[w];
  if ((int)work.size() < s->cfg.min_persistent) {
    for (auto &x : work) run_small_alone(s, w, x.first, x.second);
    return;
  }
  cudaStream_t st = sw.st;
  int64_t words = 0;
  for (auto &x : work) words += batch_words(*x.second);
  int rc0 = grow(s, sw.stage, words);
  std::vector<leiden_batch_item> items;
  std::vector<int> slot_of(work.size(), -1);
  std::vector<int64_t> nnz2(work.size(), 0);
  int64_t at = 0;
  for (size_t k = 0; k < work.size(); k++) {
    Resident *g = work[k].first;
    Request *r = work[k].second;
    r->info.graph = g->id;
    r->info.path = 0;
    if (rc0) { r->info.status = rc0; continue; }
    leiden_batch_item it{};
    it.membership_out = g->C[1 - g->mem];
    if (r->is_static) {
      it.g = csr_of(*g, g->csr, g->nnz);
      it.mode = LEIDEN_STATIC;
      nnz2[k] = g->nnz;
    } else {
      leiden_edges del{}, ins{};
      upload_batch(*r, sw.stage.buf + at, st, &del, &ins);
      at += batch_words(*r);
      const int nx = 1 - g->csr;
      leiden_csr cur = csr_of(*g, g->csr, g->nnz);
      const int rc = leiden_apply_batch(sw.ctx, &cur, &del, &ins, g->off[nx], g->idx[nx], g->w[nx], g->cap,
                                        &nnz2[k]);
      if (rc) { r->info.status = rc; continue; }
      it.g = csr_of(*g, nx, nnz2[k]);
      it.mode = s->cfg.mode;
      it.prior = g->C[g->mem];
      it.del = del;
      it.ins = ins;
    }
    slot_of[k] = (int)items.size();
    items.push_back(it);
  }
  std::vector<leiden_batch_result> res(items.size());
  int rc = LEIDEN_OK;
  if (!items.empty()) rc = leiden_batch_run(sw.batch, (int32_t)items.size(), items.data(), &s->cfg.opts,
                                            res.data());
  for (size_t k = 0; k < work.size(); k++) {
    Resident *g = work[k].first;
    Request *r = work[k].second;
    if (slot_of[k] < 0) continue;
    const leiden_batch_result &b = res[slot_of[k]];
    r->info.status = rc ? rc : b.status;
    r->info.launch_graphs = (int32_t)items.size();
    if (r->info.status == LEIDEN_OK) {
      r->info.q = b.q;
      if (!r->is_static) {
        g->csr = 1 - g->csr;
        g->nnz = nnz2[k];
      }
      g->mem = 1 - g->mem;
      g->has_aux = false;
    }
    r->info.n = g->n;
    r->info.nnz = g->nnz;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.small_launches++;
    s->st.small_graphs_launched += (int64_t)items.size();
  }
  for (auto &x : work) {
    std::vector<Request *> d{x.second};
    finish(s, x.first, d);
  }
}

// Oldest ready request among idle graphs of the given kind (lock held).
Resident *pick(leiden_server *s, bool small, const std::vector<Resident *> &taken) {
  Resident *best = nullptr;
  for (auto &kv : s->graphs) {
    Resident *g = kv.second;
    if (g->small != small || g->busy || g->queue.empty()) continue;
    if (std::find(taken.begin(), taken.end(), g) != taken.end()) continue;
    if (!best || g->queue.front()->id < best->queue.front()->id) best = g;
  }
  return best;
}

void large_worker(leiden_server *s, int k) {
  cudaSetDevice(s->device);
  for (;;) {
    Resident *g = nullptr;
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || pick(s, false, {}) != nullptr; });
      g = pick(s, false, {});
      if (!g) return;  // stopping with nothing to do
      r = g->queue.front();
      g->queue.pop_front();
      g->busy = true;
      r->t_start = Clock::now();
    }
    run_large(s, k, g, r);
  }
}

void small_worker(leiden_server *s, int wk) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<std::pair<Resident *, Request *>> work;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || pick(s, true, {}) != nullptr; });
      std::vector<Resident *> taken;
      int64_t sum_n = 0, sum_nnz = 0;
      const auto now = Clock::now();
      while ((int)work.size() < s->cfg.small_max_graphs) {
        Resident *g = pick(s, true, taken);
        if (!g) break;
        Request *r = g->queue.front();
        const int64_t nnz_after = r->is_static ? g->nnz : g->cap;
        if (!work.empty() && (sum_n + g->n > s->cfg.small_batch_n || sum_nnz + nnz_after > s->cfg.small_batch_nnz))
          break;
        sum_n += g->n;
        sum_nnz += nnz_after;
        g->queue.pop_front();
        g->busy = true;
        r->t_start = now;
        taken.push_back(g);
        work.emplace_back(g, r);
      }
      if (work.empty()) return;  // stopping with nothing to do
    }
    run_small(s, wk, work);
  }
}

void free_graph(Resident *g) {
  for (void *p : g->allocs) cudaFree(p);
  g->allocs.clear();
}

}  // namespace

extern "C" void leiden_server_config_default(leiden_server_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->hbm_budget = (int64_t)16 << 30;
  c->large_slots = 2;
  c->small_max_graphs = 64;
  c->large_max_n = (int64_t)1 << 24;
  c->large_max_nnz = (int64_t)1 << 28;
  c->small_max_n = (int64_t)1 << 16;
  c->small_max_nnz = (int64_t)1 << 18;
  c->small_batch_n = (int64_t)1 << 21;
  c->small_batch_nnz = (int64_t)1 << 24;
  c->small_workers = 2;
  c->growth = 0.25;
  c->mode = LEIDEN_DF;
  leiden_opts_default(&c->opts);
}

extern "C" int leiden_server_create(leiden_server **out, const leiden_server_config *cfg) {
  if (!out || !cfg) return LEIDEN_EINVAL;
  leiden_server_config c = *cfg;
  if (c.mode == 0) c.mode = LEIDEN_DF;
  if (c.mode != LEIDEN_DF && c.mode != LEIDEN_ND && c.mode != LEIDEN_DS) return LEIDEN_EINVAL;
  if (c.small_workers == 0) c.small_workers = 2;
  if (c.min_persistent == 0) c.min_persistent = 8;
  if (c.small_workers < 1 || c.small_workers > 8 || c.min_persistent < 1) return LEIDEN_EINVAL;
  if (c.large_slots < 1 || c.large_slots > 16 || c.small_max_graphs < 1 || c.autotune_trials < 0) return LEIDEN_EINVAL;
  if (c.hbm_budget <= 0 || c.large_max_n < 1 || c.large_max_nnz < 1 || c.small_max_n < 1 || c.small_max_nnz < 1)
    return LEIDEN_EINVAL;
  if (c.small_batch_n < c.small_max_n || c.small_batch_nnz < c.small_max_nnz || !(c.growth >= 0.0))
    return LEIDEN_EINVAL;
  if (c.opts.sched != LEIDEN_DET) return LEIDEN_EINVAL;
  leiden_server *s = new leiden_server();
  s->cfg = c;
  cudaGetDevice(&s->device);
  int rc = LEIDEN_OK;
  for (int k = 0; k < c.large_slots && !rc; k++) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { rc = LEIDEN_ECUDA; break; }
    s->large_st.push_back(st);
    leiden_ctx *ctx = nullptr;
    rc = leiden_ctx_create(&ctx, st, c.large_max_n, c.large_max_nnz);
    if (rc) break;
    s->large_ctx.push_back(ctx);
    int64_t b = 0;
    leiden_ctx_device_bytes(ctx, &b);
    s->workspace_bytes += b;
  }
  s->small.resize(c.small_workers);
  for (int k = 0; k < c.small_workers && !rc; k++) {
    leiden_server::Small &sw = s->small[k];
    if (cudaStreamCreateWithFlags(&sw.st, cudaStreamNonBlocking) != cudaSuccess) { rc = LEIDEN_ECUDA; break; }
    rc = leiden_ctx_create(&sw.ctx, sw.st, c.small_max_n, c.small_max_nnz);
    if (rc) break;
    int64_t b = 0;
    leiden_ctx_device_bytes(sw.ctx, &b);
    s->workspace_bytes += b;
    rc = leiden_batch_create(&sw.batch, sw.st, c.small_max_graphs, c.small_batch_n, c.small_batch_nnz, 0, 0);
    if (rc) break;
    leiden_batch_device_bytes(sw.batch, &b);
    s->workspace_bytes += b;
  }
  if (!rc && s->workspace_bytes > c.hbm_budget) rc = LEIDEN_ENOMEM;
  if (rc) {
    for (leiden_ctx *x : s->large_ctx) leiden_ctx_destroy(x);
    for (cudaStream_t x : s->large_st) cudaStreamDestroy(x);
    for (auto &sw : s->small) {
      if (sw.ctx) leiden_ctx_destroy(sw.ctx);
      if (sw.batch) leiden_batch_destroy(sw.batch);
      if (sw.st) cudaStreamDestroy(sw.st);
    }
    delete s;
    return rc;
  }
  s->large_stage.resize(c.large_slots);
  for (int k = 0; k < c.large_slots; k++) s->threads.emplace_back(large_worker, s, k);
  for (int k = 0; k < c.small_workers; k++) s->threads.emplace_back(small_worker, s, k);
  *out = s;
  return LEIDEN_OK;
}

extern "C" void leiden_server_destroy(leiden_server *s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [&] { return s->pending == 0; });
    s->stop = true;
    s->cv.notify_all();
  }
  for (std::thread &t : s->threads) t.join();
  for (auto &kv : s->graphs) { free_graph(kv.second); delete kv.second; }
  for (auto &kv : s->reqs) delete kv.second;
  for (leiden_ctx *x : s->large_ctx) leiden_ctx_destroy(x);
  for (cudaStream_t x : s->large_st) cudaStreamDestroy(x);
  for (Staging &sg : s->large_stage) if (sg.buf) cudaFree(sg.buf);
  for (auto &sw : s->small) {
    if (sw.stage.buf) cudaFree(sw.stage.buf);
    leiden_ctx_destroy(sw.ctx);
    leiden_batch_destroy(sw.batch);
    cudaStreamDestroy(sw.st);
  }
  delete s;
}

extern "C" int leiden_server_admit(leiden_server *s, int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx,
                                   const int32_t *w, int32_t *graph_id, int64_t *request_id) {
  if (!s || !graph_id || n < 0 || nnz < 0 || n >= INT32_MAX || !off || (nnz > 0 && (!idx || !w)))
    return LEIDEN_EINVAL;
  if (off[0] != 0 || off[n] != nnz) return LEIDEN_EINVAL;
  const int64_t cap = nnz + (int64_t)(s->cfg.growth * (double)nnz) + 1024;
  const bool small = n <= s->cfg.small_max_n && cap <= s->cfg.small_max_nnz;
  if (!small && (n > s->cfg.large_max_n || cap > s->cfg.large_max_nnz)) return LEIDEN_ENOMEM;
  const int64_t bytes = 2 * ((n + 1) * 8 + cap * 8) + 2 * (n * 4 + n * 16) + 6 * 256;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->workspace_bytes + s->resident_bytes + bytes > s->cfg.hbm_budget) return LEIDEN_ENOMEM;
    s->resident_bytes += bytes;  // reserved; released below on failure
  }
  Resident *g = new Resident();
  g->n = n;
  g->nnz = nnz;
  g->cap = cap;
  g->small = small;
  g->bytes = bytes;
  int rc = LEIDEN_OK;
  auto al = [&](void **p, size_t b) {
    if (rc) return;
    if (cudaMalloc(p, b ? b : 16) != cudaSuccess) { cudaGetLastError(); rc = LEIDEN_ENOMEM; return; }
    g->allocs.push_back(*p);
  };
  for (int k = 0; k < 2; k++) {
    al((void **)&g->off[k], (size_t)(n + 1) * 8);
    al((void **)&g->idx[k], (size_t)cap * 4);
    al((void **)&g->w[k], (size_t)cap * 4);
    al((void **)&g->C[k], (size_t)n * 4);
    al((void **)&g->K[k], (size_t)n * 8);
    al((void **)&g->Sig[k], (size_t)n * 8);
  }
  if (!rc) {
    // the caller's host arrays: plain (synchronous) copies
    if (cudaMemcpy(g->off[0], off, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        (nnz > 0 && (cudaMemcpy(g->idx[0], idx, (size_t)nnz * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                     cudaMemcpy(g->w[0], w, (size_t)nnz * 4, cudaMemcpyHostToDevice) != cudaSuccess))) {
      cudaGetLastError();
      rc = LEIDEN_ECUDA;
    }
  }
  if (rc) {
    free_graph(g);
    delete g;
    std::lock_guard<std::mutex> lk(s->mu);
    s->resident_bytes -= bytes;
    return rc;
  }
  Request *r = new Request();
  r->is_static = true;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    g->id = s->next_graph++;
    r->id = s->next_req++;
    r->graph = g->id;
    s->graphs[g->id] = g;
    s->reqs[r->id] = r;
    g->queue.push_back(r);
    s->pending++;
    s->st.resident_graphs++;
    s->cv.notify_all();
  }
  *graph_id = g->id;
  if (request_id) *request_id = r->id;
  return LEIDEN_OK;
}

extern "C" int leiden_server_submit(leiden_server *s, int32_t graph_id, const leiden_edges *del,
                                    const leiden_edges *ins, int64_t *request_id) {
  if (!s || !request_id) return LEIDEN_EINVAL;
  const int64_t nd = del ? del->count : 0, ni = ins ? ins->count : 0;
  if (nd < 0 || ni < 0) return LEIDEN_EINVAL;
  if ((nd > 0 && (!del->src || !del->dst || !del->w)) || (ni > 0 && (!ins->src || !ins->dst || !ins->w)))
    return LEIDEN_EINVAL;
  Request *r = new Request();
  if (nd) {
    r->ds.assign(del->src, del->src + nd); r->dd.assign(del->dst, del->dst + nd); r->dw.assign(del->w, del->w + nd);
  }
  if (ni) {
    r->is.assign(ins->src, ins->src + ni); r->id_.assign(ins->dst, ins->dst + ni); r->iw.assign(ins->w, ins->w + ni);
  }
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->graphs.find(graph_id);
  if (it == s->graphs.end()) { delete r; return LEIDEN_EINVAL; }
  r->id = s->next_req++;
  r->graph = graph_id;
  s->reqs[r->id] = r;
  it->second->queue.push_back(r);
  s->pending++;
  s->cv.notify_all();
  *request_id = r->id;
  return LEIDEN_OK;
}

extern "C" int leiden_server_wait(leiden_server *s, int64_t request_id, double timeout_ms, leiden_request_info *out) {
  if (!s || !out) return LEIDEN_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return LEIDEN_EINVAL;
  Request *r = it->second;
  if (timeout_ms < 0) {
    s->cv.wait(lk, [&] { return r->done; });
  } else if (!s->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] { return r->done; })) {
    return LEIDEN_ETIMEOUT;
  }
  *out = r->info;
  s->reqs.erase(it);
  delete r;
  return LEIDEN_OK;
}

namespace {
// Waits until a graph has no queued or running request (lock held).
Resident *idle_graph(leiden_server *s, std::unique_lock<std::mutex> &lk, int32_t graph_id) {
  auto it = s->graphs.find(graph_id);
  if (it == s->graphs.end()) return nullptr;
  Resident *g = it->second;
  s->cv.wait(lk, [&] { return !g->busy && g->queue.empty(); });
  return g;
}
}  // namespace

extern "C" int leiden_server_membership(leiden_server *s, int32_t graph_id, int32_t *host_out, int64_t n) {
  if (!s || (n > 0 && !host_out)) return LEIDEN_EINVAL;
  Resident *g = nullptr;
  const int32_t *src = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    g = idle_graph(s, lk, graph_id);
    if (!g || n != g->n) return LEIDEN_EINVAL;
    g->busy = true;  // no worker touches the graph while it is copied out
    src = g->C[g->mem];
  }
  int rc = LEIDEN_OK;
  if (n > 0 && cudaMemcpy(host_out, src, (size_t)n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    rc = LEIDEN_ECUDA;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  g->busy = false;
  s->cv.notify_all();
  return rc;
}

extern "C" int leiden_server_evict(leiden_server *s, int32_t graph_id) {
  if (!s) return LEIDEN_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  Resident *g = idle_graph(s, lk, graph_id);
  if (!g) return LEIDEN_EINVAL;
  s->graphs.erase(graph_id);
  s->resident_bytes -= g->bytes;
  s->st.resident_graphs--;
  free_graph(g);
  delete g;
  s->cv.notify_all();
  return LEIDEN_OK;
}

extern "C" int leiden_server_get_stats(leiden_server *s, leiden_server_stats *out) {
  if (!s || !out) return LEIDEN_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->resident_bytes = s->resident_bytes;
  out->workspace_bytes = s->workspace_bytes;
  out->budget = s->cfg.hbm_budget;
  return LEIDEN_OK;
}
