// small.h -- device-visible descriptors of the persistent many-graph kernel
// (small.cu) and the workspace layout of one graph, shared by the kernel and
// its host driver (batch.cu).
#pragma once

#include <stdint.h>

#include "leiden.h"

namespace lk {

struct SmallHeader {
  int32_t count;     // jobs in this run
  uint32_t next;     // queue head (0 at launch)
  int64_t pad[7];
};

struct SmallJob {
  int64_t n, nnz;
  const int64_t *off;
  const int32_t *idx;
  const int32_t *w;
  int32_t mode;      // LEIDEN_STATIC, LEIDEN_ND, LEIDEN_DS or LEIDEN_DF
  int32_t pad0;
  const int32_t *prior;
  int64_t nd, ni;
  const int32_t *ds, *dd, *dw, *is, *id, *iw;
  int32_t *out;
  char *ws;          // this job's workspace slice
  int64_t result;    // index of the caller's item (results are written there)
};

struct SmallOpts {
  int64_t p, q;
  double tol, tol_drop;
  int32_t max_iters, max_passes, log2S, refine_all_first_pass;
};

struct SmallResult {
  int32_t status, passes;
  int64_t affected0, changed0;
  int64_t inside, two_m;
  uint64_t sq_lo, sq_hi;
  int32_t iters[LEIDEN_STATS_PASSES];
  int64_t nv[LEIDEN_STATS_PASSES];
  int64_t nnz[LEIDEN_STATS_PASSES];
  int64_t moves[LEIDEN_STATS_PASSES];
  int64_t refine_moves[LEIDEN_STATS_PASSES];
};

// Byte offsets of one graph's arrays inside its workspace slice (every array
// 256-byte aligned).  n vertices and nnz CSR entries of the input graph bound
// every level (aggregation never grows a graph).
struct SmallLayout {
  int64_t Ctop, Cp, CB, rep, vl, pi, pc, cv, longl, gkeys, idxA, idxB, hidx;
  int64_t Kp, Sp, S2, scn, coff, ccur, hoff, cdist, offA, offB, wA, wB, hw;
  int64_t pS;
  int64_t ch, ch2, proc, stamp, flag;
  int64_t gvals;
  int log2T;         // slots of the global table: 2^log2T >= 2 n
  int64_t total;
};

__host__ __device__ inline SmallLayout small_layout(int64_t n, int64_t nnz) {
  SmallLayout L{};
  const int64_t nv = n > 0 ? n : 1;
  const int64_t ne = nnz > 0 ? nnz : 1;
  int lt = 6;
  while (((int64_t)1 << lt) < 2 * nv) lt++;
  L.log2T = lt;
  const int64_t T = (int64_t)1 << lt;
  int64_t at = 0;
  auto put = [&](int64_t bytes) {
    const int64_t o = at;
    at += (bytes + 255) & ~(int64_t)255;
    return o;
  };
  L.Ctop = put(nv * 4); L.Cp = put(nv * 4); L.CB = put(nv * 4); L.rep = put(nv * 4); L.vl = put(nv * 4);
  L.pi = put(nv * 4); L.pc = put(nv * 4); L.cv = put(nv * 4); L.longl = put(nv * 4); L.gkeys = put(T * 4);
  L.idxA = put(ne * 4); L.idxB = put(ne * 4); L.hidx = put(ne * 4);
  L.Kp = put(nv * 8); L.Sp = put(nv * 8); L.S2 = put(nv * 8); L.scn = put((nv + 1) * 8);
  L.coff = put((nv + 1) * 8); L.ccur = put(nv * 8); L.hoff = put((nv + 1) * 8); L.cdist = put((nv + 1) * 8);
  L.offA = put((nv + 1) * 8); L.offB = put((nv + 1) * 8);
  L.wA = put(ne * 8); L.wB = put(ne * 8); L.hw = put(ne * 8);
  L.pS = put(nv * 16);
  L.ch = put(nv); L.ch2 = put(nv); L.proc = put(nv); L.stamp = put(nv); L.flag = put(nv);
  L.gvals = put(T * 8);
  L.total = at;
  return L;
}

// Upper bound of small_layout(n, nnz).total that is affine in n and nnz, so
// a workspace for sum(n) vertices and sum(nnz) entries over g graphs holds
// every batch within those totals.
__host__ __device__ inline int64_t small_layout_bound(int64_t n, int64_t nnz, int64_t graphs) {
  // per vertex: 9 x 4 + 10 x 8 + 16 + 5 bytes, the global table < 4 n slots
  // of 12 bytes; per entry 3 x (4 + 8); per graph 35 arrays of alignment
  // slack, the one-element minimum of empty graphs and the 64-slot table
  return n * (36 + 80 + 16 + 5 + 48) + nnz * 36 + graphs * (35 * 256 + 1024 + 64 * 12 + 64);
}

size_t small_dyn_smem(int threads);
__global__ void small_leiden_k(SmallHeader *hdr, const SmallJob *jobs, SmallOpts o, SmallResult *results);

}  // namespace lk
