// internal.h -- host-side interface between the C-ABI driver (api.cu) and the
// kernel launchers of the other translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "leiden.h"

typedef __int128 i128;
typedef unsigned long long u64;

namespace lk {

// Every kernel launch of the library goes through LK_COUNTED, which bumps a
// process-wide counter (leiden_kernel_launches) before the launch:
//   if (n > 0) LK_COUNTED my_kernel<<<grid, block, 0, s>>>(args);
void note_launch();
#define LK_COUNTED ::lk::note_launch(),

// ---------------------------------------------------------------------------
// Degree tiers of the local-move / refinement kernels.  A vertex of degree d
// (CSR entries, self-loop included) goes to the first tier with d <= maxdeg.
// Tier 0 holds isolated vertices and is never launched.  "group" tiers give a
// vertex G lanes of a warp and an H-slot shared-memory table; "block" tiers
// give it a whole block; the last tier keeps its table in global scratch.
// ---------------------------------------------------------------------------
enum TierKind { TIER_SKIP = 0, TIER_GROUP = 1, TIER_BLOCK = 2, TIER_GLOBAL = 3 };
struct Tier {
  int kind;
  int64_t maxdeg;
  int G;        // lanes per vertex (group tiers)
  int log2H;    // table slots (group / block tiers)
  int threads;  // block size
};
static constexpr int MAX_TIERS = 12;
struct TierTable {
  int ntiers;
  Tier t[MAX_TIERS];
};
TierTable default_tiers();
// Conversions between the public tier table (leiden_tier_table) and the
// internal one (tier 0 = degree-0 vertices, never launched).
int tiers_from_public(const leiden_tier_table *p, TierTable *out);
void tiers_to_public(const TierTable &tt, leiden_tier_table *out);
// The stream a context is bound to.
cudaStream_t ctx_stream(leiden_ctx *c);

// green.cu: a green context (the primary context restricted to a share of the
// SMs).  green_push makes it current on the calling thread; green_pop undoes
// that.
struct GreenCtx {
  void *green = nullptr;  // CUgreenCtx
  void *cu = nullptr;     // CUcontext of the green context
  int sms = 0;            // SMs provisioned
};
int green_create(int device, int sm_count, GreenCtx *out);
void green_destroy(GreenCtx *g);
bool green_push(const GreenCtx &g);
void green_pop();
// Makes a context's green context current for the lifetime of the object
// (nothing for a context on the whole GPU).
struct CtxScope {
  explicit CtxScope(leiden_ctx *c);
  ~CtxScope();
  bool pushed = false;
};

template <typename WT>
struct GraphView {
  int64_t n;
  const int64_t *off;
  const int32_t *idx;
  const WT *w;
};

// Arguments of the local-move and refinement kernels (Alg. leidenlm,
// Alg. leidenre).  Scores are Eq. 2 scaled by 2m^2 q:
//   S = A (K_{i->c} - K_{i->d}) - p K_i (K_i + Sigma_c - Sigma_d),  A = 2m q.
template <typename WT>
struct MoveArgs {
  GraphView<WT> g;
  const int32_t *list;   // vertices of one (class, tier) bucket
  int64_t list_n;
  int32_t *C;            // C'
  const int64_t *K;      // K'
  int64_t *Sig;          // Sigma'
  uint8_t *processed;    // vertex pruning flags (local-move)
  const uint8_t *in_range;  // DS affected range in pass 0, else NULL
  const int32_t *CB;     // community bounds (refinement)
  uint8_t *changed;      // Delta C'
  uint8_t *stamp;        // refinement: sub-sweep in which a vertex proposed
  uint8_t stamp_val;
  int dynamic;           // mark changed communities on migration
  int spec;              // most listed vertices are eligible: load their headers
                         // alongside the eligibility test, not after it
  int32_t *prop_i;       // DET proposals
  int32_t *prop_c;
  i128 *prop_S;
  u64 *prop_count;
  int64_t A;             // 2m * q
  int64_t p;
  int32_t *gkeys;        // global scratch tables (hub rows); all keys empty and
  u64 *gvals;            // all values zero whenever no kernel is using them
  int glog2H;
  int gblocks;
  int32_t *big;          // movers whose rows are re-marked by the big-row kernel
  u64 *ctr;              // counters, see CTR_*
};

// Work arrays of the multi-block hub path (hub.cu), indexed by the position
// of the hub in its (class, tier) list.
struct HubWork {
  int64_t *tsz;   // table slots (0: hub not eligible)
  int64_t *toff;  // exclusive scan of tsz
  int64_t *ioff;  // exclusive scan of insert work items
  int64_t *soff;  // exclusive scan of scan work items
  int64_t *tot;   // [0] table slots, [1] insert items, [2] scan items
  i128 *psc;      // per scan item: best partial score,
  int32_t *pc;    //   its community,
  int64_t *pkid;  //   and the weight towards the hub's own community
};
static constexpr int64_t HUB_TABLE_MIN = 4096;
// Build-time tunables.  LK_AGG_ROUND_SLOTS / LK_HUB_ROUND_SLOTS cap the
// global hash-table slots (12 B each) processed per round of the aggregation
// and hub kernels (0: only the scratch capacity limits a round); a cap near
// 6 Mi keeps a round's tables resident in L2.  LK_AUX_STREAMS is the number of
// auxiliary streams the tier kernels of a sub-sweep fan out to (0: all on the
// context stream).
#ifndef LK_AGG_ROUND_SLOTS
#define LK_AGG_ROUND_SLOTS 0
#endif
#ifndef LK_HUB_ROUND_SLOTS
#define LK_HUB_ROUND_SLOTS 0
#endif
// 1: hub rows with at most 64 Ki distinct candidates are decided by a thread-
// block cluster with the table in distributed shared memory (0: every hub row
// through the global-memory tables).  Same decisions either way; measured
// slower on Chung-Lu (3.33 against 2.92 s per Static) and R-MAT scale 22 (170
// against 149 ms): a cluster holds eight SMs per hub and the other degree
// tiers of the colour class wait for them.
#ifndef LK_HUB_CLUSTERS
#define LK_HUB_CLUSTERS 0
#endif
// 1: every level compares candidate scores in 128 bits, whatever its
// largest K' (a testing aid: both widths must give the same decisions).
#ifndef LK_FORCE_WIDE_SCORES
#define LK_FORCE_WIDE_SCORES 0
#endif
#ifndef LK_AUX_STREAMS
#define LK_AUX_STREAMS 6
#endif
// Table slots and row entries each lane of a decide kernel keeps in flight.
// Measured on R-MAT scale 22 (Static, DET): 1/1 is fastest; unrolling the
// gathers raises registers and lowers occupancy more than it hides latency.
#ifndef LK_SCAN_UNROLL
#define LK_SCAN_UNROLL 1
#endif
#ifndef LK_ROW_UNROLL
#define LK_ROW_UNROLL 1
#endif
// Neighbour re-marking of the DET apply: row entries per lane in flight.
#ifndef LK_REMARK_UNROLL
#define LK_REMARK_UNROLL 4
#endif
// Row entries per lane in flight in the block-tier decide kernel.
#ifndef LK_BLOCK_ROW_UNROLL
#define LK_BLOCK_ROW_UNROLL 4
#endif
// 32-entry chunks of a hub row a warp loads before it inserts them (their
// row loads, C'[j] gathers and first table probes all in flight together).
// Row entries of one hub-insert work item.
#ifndef LK_HUB_CHUNK
#define LK_HUB_CHUNK 4096
#endif
// Movers with rows longer than this re-mark their neighbours through the
// big-row kernel (spread over many blocks) instead of half a warp.
#ifndef LK_BIG_ROW
#define LK_BIG_ROW 4096
#endif
#ifndef LK_HUB_UNROLL
#define LK_HUB_UNROLL 1
#endif
// Resident blocks per SM the group-tier decide kernels are compiled for (a
// register cap for 256-thread blocks); 0 leaves the register count to the
// compiler.
#ifndef LK_GROUP_MINB
#define LK_GROUP_MINB 0
#endif


enum {
  CTR_SCANNED_ENTRIES = 0,
  CTR_SCANNED_VERTICES = 1,
  CTR_CANDIDATES = 2,
  CTR_SUMS_LO = 3,      // i128 sum of S over applied moves (lo, hi)
  CTR_SUMS_HI = 4,
  CTR_MOVES = 5,
  CTR_PROPS = 6,        // proposal count of the current sub-sweep
  CTR_ERROR = 7,
  CTR_NCOMM = 8,
  CTR_SCRATCH0 = 9,     // 9..12: scratch words of the host driver
  CTR_BIG = 13,         // movers appended to the big-row list
  CTR_COUNT = 16
};

// move.cu
template <typename WT, typename ST, bool REFINE, bool ASYNC>
void launch_decide(const Tier &tier, const MoveArgs<WT> &a, int sms, cudaStream_t s);
void launch_apply_moves(const int32_t *prop_i, const int32_t *prop_c, const i128 *prop_S,
                        u64 *ctr, int32_t *C, const int64_t *K, int64_t *Sig,
                        uint8_t *changed, uint8_t *processed, const int64_t *off,
                        const int32_t *idx, int32_t *big, int dynamic, int sms, cudaStream_t s);
// Movers with more than BIG_ROW entries leave their neighbour re-marking
// to launch_mark_big, which spreads each row over the whole grid.
static constexpr int64_t BIG_ROW = LK_BIG_ROW;
void launch_mark_big(const int32_t *big, const u64 *count, const int64_t *off, const int32_t *idx,
                     uint8_t *processed, int sms, cudaStream_t s);
// hub.cu
template <typename WT, typename ST, bool REFINE, bool ASYNC>
void launch_hubs(const MoveArgs<WT> &a, const HubWork &hw, int sms, cudaStream_t s);
void launch_apply_refine(const int32_t *prop_i, const int32_t *prop_c, u64 *ctr,
                         const uint8_t *stamp, uint8_t sv, int32_t *C, const int64_t *K,
                         int64_t *Sig, int sms, cudaStream_t s);

// buckets.cu
// Builds the vertex lists of every (class, tier) key, key = class * ntiers + tier,
// stored key-major in `list`; koff_dev[key] / koff_dev[nkeys] are the offsets.
void launch_buckets(const int64_t *off, int64_t n, int log2S, const TierTable &tt,
                    int32_t *list, int32_t *blockhist, int64_t *scanned, int64_t *koff_dev,
                    int64_t *scan_tmp, cudaStream_t s);
int64_t bucket_blockhist_elems(int64_t n, int nkeys);

// scan.cu
void ensure_smem(const void *func, size_t bytes);
// Blocks of `func` (threads, dynamic shared memory) resident at once on `sms`
// SMs: the grid of a grid-stride kernel that leaves no partial last wave.
int64_t resident_blocks(const void *func, int threads, size_t smem, int sms);
template <typename TI>
void exclusive_scan(const TI *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);

// misc.cu
template <typename WT>
void launch_row_sums(GraphView<WT> g, int64_t *K, cudaStream_t s);
void launch_iota(int32_t *a, int64_t n, cudaStream_t s);
void launch_fill_u8(uint8_t *a, uint8_t v, int64_t n, cudaStream_t s);
void launch_copy_i64(int64_t *dst, const int64_t *src, int64_t n, cudaStream_t s);
void launch_invert_u8(uint8_t *dst, const uint8_t *src, int64_t n, cudaStream_t s);
void launch_clear_left(int64_t *Sig, int64_t n, cudaStream_t s);
void launch_sum_i64(const int64_t *a, int64_t n, u64 *out, cudaStream_t s);
void launch_subset_renumber(int64_t n, int32_t *C, const int64_t *Sig, int64_t *Sig2,
                            const uint8_t *ch, uint8_t *ch2, int32_t *rep, cudaStream_t s);
void launch_break(int64_t n, int32_t *C, const int64_t *K, int64_t *Sig, const uint8_t *ch,
                  cudaStream_t s);
// dense renumbering; returns |Gamma| in ctr[CTR_NCOMM] (device)
void launch_renumber(int64_t n, int32_t *C, uint8_t *exists, int64_t *scanned, int64_t *tmp,
                     u64 *ctr, cudaStream_t s);
void launch_lookup(int64_t n, int32_t *Ctop, const int32_t *Cp, cudaStream_t s);
void launch_canonical(int64_t n, const int32_t *C, int32_t *out, int32_t *minv, uint8_t *flag,
                      int64_t *scanned, int64_t *tmp, cudaStream_t s);
// Eq. 1 terms of membership C on g (nnz entries): acc[0] internal weight,
// acc[1..2] sum of Sigma_c^2 (i128), acc[3] 2m.  Bounds-checked: a bad row,
// label or column ID is skipped and sets 512 in *err; nothing runs when *err
// is already set.
template <typename WT>
void launch_modularity_terms(GraphView<WT> g, int64_t nnz, const int32_t *C, int64_t *Sig_tmp, u64 *acc,
                             u64 *err, cudaStream_t s);
void launch_update_weights(int64_t count, const int32_t *src, const int32_t *dst,
                           const int32_t *w, int sign, const int32_t *Cprev, int64_t *K,
                           int64_t *Sig, cudaStream_t s);
void launch_changed_communities(int64_t count, const int32_t *src, const int32_t *dst,
                                const int32_t *Cprev, uint8_t *changed, cudaStream_t s);
void launch_mark_df(int64_t count, const int32_t *src, const int32_t *dst, const int32_t *Cprev,
                    int same, uint8_t *affected, cudaStream_t s);
void launch_check_ids(int64_t count, const int32_t *src, const int32_t *dst, const int32_t *w,
                      int64_t n, u64 *err, cudaStream_t s);
void launch_check_graph(int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx, const int32_t *w,
                        u64 *err, cudaStream_t s);
void launch_check_range(const int32_t *a, int64_t n, int64_t hi, u64 *err, cudaStream_t s);
void launch_sigma_from(int64_t n, const int32_t *C, const int64_t *K, int64_t *Sig,
                       cudaStream_t s);

// agg.cu: Alg. leidenag.  Input level graph g (nc communities in dense C);
// output CSR (off2[nc+1], idx2, w2); returns nnz via ctr[CTR_SCRATCH0].
struct AggWork {
  int64_t *ccount, *coff, *ctdeg, *hoff, *cdist, *off2tmp;
  int64_t *ccur;
  int32_t *cv, *clist;
  int32_t *hidx;
  int64_t *hw;
  int32_t *gkeys;
  u64 *gvals;
  int64_t gcap;
  int32_t *blockhist;
  int64_t *scanned;
  int64_t *koff_dev;
  int64_t *scan_tmp;
  int64_t *h_koff;       // pinned host, >= MAX_TIERS + 3 entries
  int64_t *Kout;         // [nc] row sums of the super-vertex graph (its K')
  u64 *bcnt;             // [bcap] giant-community bucket counters
  int64_t *bpos;         // [bcap] bucket offsets in the scratch arrays
  int64_t bcap;
  u64 *ctr;
  int sms;
  int uniform;           // 1: every community through the multi-block path
};
template <typename WT>
int aggregate(GraphView<WT> g, const int32_t *C, int64_t nc, int64_t *off2, int32_t *idx2,
              int64_t *w2, int64_t *nnz2, const AggWork &wk, cudaStream_t s);

// ds.cu / batch.cu
struct DsWork {
  int64_t *cnt;      // [n+1]
  int64_t *soff;     // [n+1]
  int64_t *cur;      // [n]
  int32_t *sdst;     // [2*ni]
  int32_t *swt;      // [2*ni]
  int64_t *scan_tmp;
  uint8_t *dE, *dC;
};
void launch_mark_ds(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *Cprev,
                    const int64_t *K, const int64_t *Sig, int64_t A, int64_t p,
                    int64_t nd, const int32_t *ds, const int32_t *dd,
                    int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw,
                    uint8_t *affected, const DsWork &wk, cudaStream_t s);

struct BatchWork {
  int64_t *cnt;      // [n+1] updates per row, then merged records per touched row
  int64_t *uoff;     // [n+1] exclusive scan of the update counts
  int64_t *cur;      // [n+1]
  int32_t *ut;       // [2*(nd+ni)] update targets, by row
  int32_t *uw;       // [2*(nd+ni)] signed weights (deletions negative), then new weights
  uint8_t *uk;       // [2*(nd+ni)] record kinds
  int32_t *Rp, *Np;  // [2*(nd+ni)] removed / new entries before each record of its row
  uint8_t *tflag;    // [n+1] touched rows
  int64_t *tpos;     // [n+1] their exclusive scan
  int32_t *trow;     // [n] touched rows in increasing order
  int64_t *newdeg;   // [n+1]
  uint32_t *bits;    // [nnz/32 + 1] row starts
  int64_t *scan_tmp;
  u64 *err;
};
int apply_batch(int64_t n, const int64_t *off, const int32_t *idx, const int32_t *w,
                int64_t nd, const int32_t *ds, const int32_t *dd, const int32_t *dw,
                int64_t ni, const int32_t *is, const int32_t *id, const int32_t *iw,
                int64_t *off_out, int32_t *idx_out, int32_t *w_out, int64_t cap_nnz,
                int64_t *nnz_out, const BatchWork &wk, cudaStream_t s);

}  // namespace lk
