// tune.cu -- the public tier table (leiden_tier_table), its validation, and
// the autotuner that picks a table per graph by timing candidates.
//
// The tier table only decides which kernel shape processes a vertex of a
// given degree (lanes per vertex, hashtable slots, block size, and where the
// multi-block hub path starts); every shape computes the same decision for
// the same vertex, so the tuner can compare candidates on time alone.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "leiden.h"

namespace lk {

namespace {

constexpr int64_t kSmemPerBlock = 227 * 1024;
constexpr int64_t kSlotBytes = 12;              // u64 value + int32 key
constexpr int64_t kGroupStaticSmem = 8 * 32 * 8;   // decide_group's combine scratch
constexpr int64_t kBlockStaticSmem = 10 * 1024;    // decide_block's scratch, rounded up

bool group_shape_supported(int lanes, int log2_slots) {
  switch (lanes) {
    case 1: return log2_slots == 2 || log2_slots == 3;   // one lane, 4 or 8 entries in registers
    case 4: return log2_slots == 3 || log2_slots == 4;
    case 8: return log2_slots == 4 || log2_slots == 5;
    case 16: return log2_slots == 5 || log2_slots == 6;
    case 32: return log2_slots >= 6 && log2_slots <= 10;
    default: return false;
  }
}

}  // namespace

int tiers_from_public(const leiden_tier_table *p, TierTable *out) {
  if (leiden_tiers_validate(p) != LEIDEN_OK) return LEIDEN_EINVAL;
  TierTable tt{};
  tt.t[0] = {TIER_SKIP, 0, 0, 0, 0};
  for (int k = 0; k < p->count; k++) {
    const leiden_tier &s = p->tier[k];
    Tier &d = tt.t[k + 1];
    if (s.kind == LEIDEN_TIER_GROUP) d = {TIER_GROUP, s.max_degree, s.lanes, s.log2_slots, s.threads};
    else if (s.kind == LEIDEN_TIER_BLOCK) d = {TIER_BLOCK, s.max_degree, 0, s.log2_slots, s.threads};
    else d = {TIER_GLOBAL, INT64_MAX, 0, 0, 1024};
  }
  tt.ntiers = p->count + 1;
  *out = tt;
  return LEIDEN_OK;
}

void tiers_to_public(const TierTable &tt, leiden_tier_table *out) {
  memset(out, 0, sizeof(*out));
  out->count = tt.ntiers - 1;
  for (int k = 1; k < tt.ntiers && k - 1 < LEIDEN_MAX_TIERS; k++) {
    const Tier &s = tt.t[k];
    leiden_tier &d = out->tier[k - 1];
    if (s.kind == TIER_GROUP) d = {LEIDEN_TIER_GROUP, s.G, s.log2H, s.threads, s.maxdeg};
    else if (s.kind == TIER_BLOCK) d = {LEIDEN_TIER_BLOCK, 0, s.log2H, s.threads, s.maxdeg};
    else d = {LEIDEN_TIER_HUB, 0, 0, 0, INT64_MAX};
  }
}

}  // namespace lk

using namespace lk;

extern "C" void leiden_tiers_default(leiden_tier_table *out) {
  if (out) tiers_to_public(default_tiers(), out);
}

extern "C" int leiden_tiers_validate(const leiden_tier_table *t) {
  if (!t || t->count < 1 || t->count > LEIDEN_MAX_TIERS || t->reserved != 0) return LEIDEN_EINVAL;
  int64_t prev = 0;
  for (int k = 0; k < t->count; k++) {
    const leiden_tier &s = t->tier[k];
    const bool last = k == t->count - 1;
    if (s.kind == LEIDEN_TIER_HUB) {
      if (!last || s.lanes != 0 || s.log2_slots != 0 || s.threads != 0) return LEIDEN_EINVAL;
      continue;
    }
    if (last) return LEIDEN_EINVAL;  // the hub tier must close the table
    if (s.max_degree <= prev) return LEIDEN_EINVAL;
    prev = s.max_degree;
    if (s.threads % 32 != 0) return LEIDEN_EINVAL;
    if (s.kind == LEIDEN_TIER_GROUP) {
      if (!group_shape_supported(s.lanes, s.log2_slots)) return LEIDEN_EINVAL;
      if (s.threads < 32 || s.threads > 256) return LEIDEN_EINVAL;
      const int64_t smem = (int64_t)(s.threads / 32) * (32 / s.lanes) * ((int64_t)1 << s.log2_slots) * kSlotBytes;
      if (smem + kGroupStaticSmem > kSmemPerBlock) return LEIDEN_EINVAL;
    } else if (s.kind == LEIDEN_TIER_BLOCK) {
      if (s.lanes != 0 || s.log2_slots < 6 || s.log2_slots > 14) return LEIDEN_EINVAL;
      if (s.threads < 64 || s.threads > 1024) return LEIDEN_EINVAL;
      // 12 bytes per slot plus a 2-byte used-slot list of half the table
      if (((int64_t)1 << s.log2_slots) * (kSlotBytes + 1) + kBlockStaticSmem > kSmemPerBlock) return LEIDEN_EINVAL;
    } else {
      return LEIDEN_EINVAL;
    }
    // a row never fills its table past half: 2^log2_slots >= 2 * degree; a
    // one-lane tier holds the whole row in 2^log2_slots registers
    if (s.kind == LEIDEN_TIER_GROUP && s.lanes == 1) {
      if (((int64_t)1 << s.log2_slots) < s.max_degree) return LEIDEN_EINVAL;
    } else if (((int64_t)1 << s.log2_slots) < 2 * s.max_degree) {
      return LEIDEN_EINVAL;
    }
  }
  return LEIDEN_OK;
}

// ---------------------------------------------------------------------------
// Autotuner.
// ---------------------------------------------------------------------------
namespace {

leiden_tier G(int lanes, int log2_slots, int threads, int64_t maxdeg) {
  return {LEIDEN_TIER_GROUP, lanes, log2_slots, threads, maxdeg};
}
leiden_tier B(int log2_slots, int threads, int64_t maxdeg) {
  return {LEIDEN_TIER_BLOCK, 0, log2_slots, threads, maxdeg};
}
leiden_tier HUB() { return {LEIDEN_TIER_HUB, 0, 0, 0, INT64_MAX}; }

leiden_tier_table make(std::initializer_list<leiden_tier> ts) {
  leiden_tier_table t{};
  for (const leiden_tier &x : ts) t.tier[t.count++] = x;
  return t;
}

// Candidate tables, the default first, then variants of one or two choices
// each: hashtable load (tables 4x the row instead of 2x), block shapes of the
// group tiers, the split between warp groups and whole blocks for rows of
// 129..512 entries, the block sizes of the block tiers, and where the hub
// path starts.
std::vector<leiden_tier_table> candidates() {
  std::vector<leiden_tier_table> v;
  leiden_tier_table d{};
  leiden_tiers_default(&d);
  v.push_back(d);
  // warp groups of 4 and 8 lanes with shared tables for the shortest rows
  v.push_back(make({G(4, 3, 256, 4), G(8, 4, 256, 8), G(16, 5, 256, 16), G(32, 6, 256, 32), G(32, 8, 256, 128),
                    G(32, 9, 256, 256), B(10, 128, 512), B(12, 256, 2048), B(14, 512, 8192), HUB()}));
  // sparser tables for short rows (fewer probe collisions)
  v.push_back(make({G(4, 4, 256, 4), G(8, 5, 256, 8), G(16, 6, 256, 16), G(32, 7, 256, 32), G(32, 9, 256, 128),
                    G(32, 10, 128, 512), B(12, 256, 2048), B(14, 512, 8192), HUB()}));
  // smaller blocks for the group tiers (more blocks resident per SM)
  v.push_back(make({G(4, 3, 128, 4), G(8, 4, 128, 8), G(16, 5, 128, 16), G(32, 6, 128, 32), G(32, 8, 128, 128),
                    G(32, 10, 64, 512), B(12, 256, 2048), B(14, 512, 8192), HUB()}));
  // rows of 129..512 entries on whole blocks instead of one warp each
  v.push_back(make({G(4, 3, 256, 4), G(8, 4, 256, 8), G(16, 5, 256, 16), G(32, 6, 256, 32), G(32, 8, 256, 128),
                    B(10, 128, 512), B(12, 256, 2048), B(14, 512, 8192), HUB()}));
  // wider lanes for the shortest rows (no 4-lane groups)
  v.push_back(make({G(8, 4, 256, 8), G(16, 5, 256, 16), G(32, 6, 256, 32), G(32, 8, 256, 128), G(32, 10, 128, 512),
                    B(12, 256, 2048), B(14, 512, 8192), HUB()}));
  // larger blocks for the block tiers
  v.push_back(make({G(4, 3, 256, 4), G(8, 4, 256, 8), G(16, 5, 256, 16), G(32, 6, 256, 32), G(32, 8, 256, 128),
                    G(32, 10, 128, 512), B(12, 512, 2048), B(14, 1024, 8192), HUB()}));
  // hub path from 2048 entries
  v.push_back(make({G(4, 3, 256, 4), G(8, 4, 256, 8), G(16, 5, 256, 16), G(32, 6, 256, 32), G(32, 8, 256, 128),
                    G(32, 10, 128, 512), B(12, 256, 2048), HUB()}));
  // finer degree steps between 32 and 512
  v.push_back(make({G(4, 3, 256, 4), G(8, 4, 256, 8), G(16, 5, 256, 16), G(32, 6, 256, 32), G(32, 7, 256, 64),
                    G(32, 8, 256, 128), G(32, 9, 256, 256), G(32, 10, 128, 512), B(12, 256, 2048), B(14, 512, 8192),
                    HUB()}));
  // smaller blocks everywhere
  v.push_back(make({G(4, 3, 128, 4), G(8, 4, 128, 8), G(16, 5, 128, 16), G(32, 6, 128, 32), G(32, 8, 128, 128),
                    B(10, 128, 512), B(12, 128, 2048), B(14, 256, 8192), HUB()}));
  return v;
}

}  // namespace

extern "C" int leiden_autotune(leiden_ctx *ctx, const leiden_csr *g, const leiden_opts *opts, int32_t max_trials,
                               int32_t repeats, leiden_tier_table *best_out, double *best_ms) {
  if (!ctx || !g || max_trials < 1 || repeats < 1) return LEIDEN_EINVAL;
  CtxScope scope(ctx);  // the timing events belong to the context's (green) context
  cudaStream_t st = ctx_stream(ctx);
  leiden_tier_table keep{};
  leiden_ctx_get_tiers(ctx, &keep);
  int32_t *memb = nullptr;
  if (g->n > 0 && cudaMalloc(&memb, (size_t)g->n * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    return LEIDEN_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<leiden_tier_table> cand = candidates();
  if ((int)cand.size() > max_trials) cand.resize(max_trials);
  int rc = LEIDEN_OK;
  int best = -1;
  double best_t = 0.0;
  for (size_t k = 0; k < cand.size() && rc == LEIDEN_OK; k++) {
    rc = leiden_ctx_set_tiers(ctx, &cand[k]);
    if (rc) break;
    std::vector<double> ts;
    for (int r = 0; r < repeats && rc == LEIDEN_OK; r++) {
      cudaEventRecord(e0, st);
      rc = leiden_static(ctx, g, opts, memb, nullptr);
      cudaEventRecord(e1, st);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = LEIDEN_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ts.push_back(ms);
    }
    if (rc) break;
    std::sort(ts.begin(), ts.end());
    const double med = ts[ts.size() / 2];
    if (best < 0 || med < best_t) { best = (int)k; best_t = med; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (memb) cudaFree(memb);
  if (rc || best < 0) {
    leiden_ctx_set_tiers(ctx, &keep);
    return rc ? rc : LEIDEN_EINVAL;
  }
  leiden_ctx_set_tiers(ctx, &cand[best]);
  if (best_out) *best_out = cand[best];
  if (best_ms) *best_ms = best_t;
  return LEIDEN_OK;
}
