/*
 * leiden.h -- C-ABI of the GB300 (sm_103a) library for Static, Naive-dynamic
 * (ND), Delta-screening (DS) and Dynamic Frontier (DF) Leiden community
 * detection (arXiv 2405.11658).
 *
 * Problem statement (Sec. 3.5, Sec. 4.5, Appendix A): Static Leiden maps a
 * graph G to a community membership C; a dynamic update takes the updated
 * snapshot G^t, the batch of edge deletions D- and insertions D+ that produced
 * it, the previous membership C^{t-1}, weighted degrees K^{t-1} and community
 * totals Sigma^{t-1}, and returns C^t, K^t and Sigma^t.
 *
 * General conventions
 *   - All graph, batch and output arrays are DEVICE pointers owned by the
 *     caller, unless a field says HOST.  The library never frees them.
 *   - A graph is a symmetric CSR without duplicate entries: off[n+1] (int64,
 *     off[0] = 0), idx[nnz] (int32 column IDs in [0, n)), w[nnz] (int32, > 0).
 *     A self-loop (i,i,w) is stored once and adds w to K_i and to 2m (Sec. 3
 *     definitions of K_i and m).  Rows need not be sorted, except for
 *     leiden_apply_batch (below).
 *   - A batch lists each undirected pair once, (src, dst, w); the library
 *     applies both directions, as every update carries its reverse edge
 *     (Sec. 5.1.4).  Self-loops are rejected.
 *   - Membership outputs are canonical: the community holding the smallest
 *     vertex is 0, the next smallest unseen vertex opens community 1, and so on.
 *   - Every call is ordered on the context's CUDA stream.  Calls that return a
 *     host scalar (q_out, nnz_out) or read sizes back synchronise that stream.
 *   - Return value: LEIDEN_OK (0) or a negative LEIDEN_E* code.  On error,
 *     outputs are unspecified (the library may have written part of them);
 *     the context stays usable unless the code is LEIDEN_ECUDA.
 *   - Integer arithmetic is exact: K and Sigma in int64, the delta-modularity
 *     of Eq. 2 scaled by 2m^2 q in 128-bit integers.  The resolution gamma
 *     must be an exact multiple of 2^-20 (gamma = p/q, q = 2^20), else
 *     LEIDEN_EINVAL.  2m must stay below 2^40 (else LEIDEN_EOVERFLOW).
 */
#ifndef LEIDEN_H
#define LEIDEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LEIDEN_OK 0
#define LEIDEN_EINVAL (-1)     /* bad argument, bad ID, bad batch, bad gamma */
#define LEIDEN_ENOMEM (-2)     /* a size exceeds the context's capacity, or allocation failed */
#define LEIDEN_EOVERFLOW (-3)  /* 2m >= 2^40 */
#define LEIDEN_ETIMEOUT (-4)   /* a bounded device wait expired */
#define LEIDEN_ECUDA (-5)      /* a CUDA call failed; the context should be destroyed */

typedef struct {
  int64_t n;            /* vertices, 0 <= n < 2^31 */
  int64_t nnz;          /* CSR entries (= off[n]) */
  const int64_t *off;   /* DEVICE [n+1] */
  const int32_t *idx;   /* DEVICE [nnz] */
  const int32_t *w;     /* DEVICE [nnz], > 0 */
} leiden_csr;

typedef struct {
  int64_t count;        /* undirected pairs */
  const int32_t *src;   /* DEVICE [count] */
  const int32_t *dst;   /* DEVICE [count] */
  const int32_t *w;     /* DEVICE [count], > 0; for a deletion, the weight of the deleted edge */
} leiden_edges;

enum { LEIDEN_ND = 1, LEIDEN_DS = 2, LEIDEN_DF = 3 };

/* Schedules.  Both walk det_subsets colour classes in order in every
 * local-move iteration and in the refinement sweep (class(i) = top log2(S)
 * bits of (uint32)(i * 2654435761)).  DET: the moves of a class are chosen
 * against the state at its start and applied together, so the result does
 * not depend on thread timing.  ASYNC: inside a class, vertices move in place
 * as soon as they decide, as in the paper's asynchronous CPU implementation
 * (Sec. 4.7); the class's degree tiers run from the longest rows down, and a
 * vertex alone in its community joins another singleton only if that one has
 * the smaller label (Lu, Halappanavar and Kalyanaraman 2015); results vary
 * with timing. */
enum { LEIDEN_DET = 0, LEIDEN_ASYNC = 1 };

typedef struct {
  double gamma;                  /* resolution (1.0) */
  double tol;                    /* initial iteration tolerance tau (0.01, Sec. 4.7) */
  double tol_drop;               /* tau divisor per pass (10, Sec. 4.7) */
  int32_t max_iters;             /* MAX_ITERATIONS per local-moving phase (20, Sec. 4.7) */
  int32_t max_passes;            /* MAX_PASSES (10; not stated by the paper) */
  int32_t sched;                 /* LEIDEN_DET or LEIDEN_ASYNC */
  int32_t det_subsets;           /* DET colour classes: power of two in [1, 256] (8) */
  int32_t refine_all_first_pass; /* Full Refine variant (Sec. 4.2): refine every community in pass 0 */
  int32_t reserved[3];           /* must be 0 */
} leiden_opts;

/* Fills the defaults listed above. */
void leiden_opts_default(leiden_opts *opts);

typedef struct leiden_ctx leiden_ctx;

/* Creates a context bound to one CUDA stream (cudaStream_t passed as void*;
 * NULL = the legacy default stream) on the current device, and allocates its
 * device workspace for graphs of up to max_n vertices and max_nnz CSR entries
 * (about 100 B per vertex plus 52 B per entry).  The stream is borrowed and
 * must outlive the context.  Errors: LEIDEN_EINVAL (sizes out of range),
 * LEIDEN_ENOMEM, LEIDEN_ECUDA. */
int leiden_ctx_create(leiden_ctx **out, void *cuda_stream, int64_t max_n, int64_t max_nnz);

/* Creates a context restricted to a share of the GPU's SMs: a green context
 * (the current device's primary context with at least sm_count SMs
 * provisioned; the driver rounds the count up to its partition granularity,
 * 8 SMs on this architecture), a non-blocking stream inside it that the
 * context owns, and the workspace of leiden_ctx_create.  Every kernel the
 * context launches runs on those SMs only, and grids are sized for them; the
 * results are the same as on the whole GPU.  This is the GPU counterpart of
 * running the paper's implementation on fewer threads (Sec. 5.2, strong
 * scaling).  Device memory stays shared with the primary context, so graphs
 * allocated elsewhere on the device can be passed in.  sms_granted (HOST, may
 * be NULL) receives the SM count provisioned.  Every call on the context makes
 * the green context current on the calling thread for its duration.  Errors:
 * LEIDEN_EINVAL (sm_count outside [1, SM count], sizes out of range),
 * LEIDEN_ENOMEM, LEIDEN_ECUDA (green contexts unavailable). */
int leiden_ctx_create_sm(leiden_ctx **out, int32_t sm_count, int64_t max_n, int64_t max_nnz,
                         int32_t *sms_granted);

/* The number of SMs the context sizes its grids for (HOST out). */
int leiden_ctx_sm_count(leiden_ctx *ctx, int32_t *out);

/* Synchronises the stream and frees the workspace (and, for a context from
 * leiden_ctx_create_sm, its stream and green context).  NULL is a no-op. */
void leiden_ctx_destroy(leiden_ctx *ctx);

/* Static Leiden (Alg. leiden with every vertex affected and every community
 * changed, Sec. 4.6): membership_out DEVICE [n] receives canonical labels;
 * q_out (HOST, may be NULL) receives the modularity of Eq. 1 at resolution
 * gamma.  Errors: LEIDEN_EINVAL, LEIDEN_ENOMEM (n or nnz above the context's
 * capacity), LEIDEN_EOVERFLOW, LEIDEN_ECUDA. */
int leiden_static(leiden_ctx *ctx, const leiden_csr *g, const leiden_opts *opts,
                  int32_t *membership_out, double *q_out);

/* ND / DS / DF update (Alg. naive, Alg. delta, Alg. frontier with
 * Alg. update and Alg. leiden).  g_t is the updated snapshot G^t, already
 * containing the batch (see leiden_apply_batch); del / ins is the batch that
 * produced it (either may be NULL or empty).  prior_membership DEVICE [n]
 * holds C^{t-1} (any labels in [0, n)); prior_K and prior_Sigma DEVICE [n]
 * hold K^{t-1} and Sigma^{t-1} indexed by those labels, or are both NULL, in
 * which case K^t and Sigma^t are recomputed from G^t.  Outputs (DEVICE [n]):
 * canonical C^t, K^t, and Sigma^t indexed by the canonical labels of C^t
 * (zero beyond the last community); K_out, Sigma_out and q_out may be NULL.
 * mode: LEIDEN_ND, LEIDEN_DS or LEIDEN_DF.  Errors as leiden_static, plus
 * LEIDEN_EINVAL for a bad mode or batch IDs outside [0, n). */
int leiden_update(leiden_ctx *ctx, const leiden_csr *g_t,
                  const int32_t *prior_membership, const int64_t *prior_K,
                  const int64_t *prior_Sigma, const leiden_edges *del,
                  const leiden_edges *ins, int32_t mode, const leiden_opts *opts,
                  int32_t *membership_out, int64_t *K_out, int64_t *Sigma_out,
                  double *q_out);

/* Modularity (Eq. 1 at resolution gamma) of membership (DEVICE [n], labels
 * in [0, n)) on g.  q_out is HOST.  The graph and the labels are validated
 * on the device, and the verdict read, before any kernel indexes by them.
 * Errors: LEIDEN_EINVAL (malformed graph, label out of range, bad gamma),
 * LEIDEN_ENOMEM, LEIDEN_EOVERFLOW (nnz > 2^32 or 2m >= 2^40), LEIDEN_ECUDA. */
int leiden_modularity(leiden_ctx *ctx, const leiden_csr *g, const int32_t *membership,
                      double gamma, double *q_out);

/* Builds G^t = G^{t-1} - D- + D+ (Sec. 3.5) on the device.  g_prev must have
 * sorted rows; the output rows are sorted.  A deletion removes the edge
 * {src, dst}; it must exist with weight w.  Deletions apply before insertions;
 * an insertion of an existing (or repeated) pair adds its weight.  off_out
 * DEVICE [n+1], idx_out / w_out DEVICE [cap_nnz]; nnz_out (HOST) receives the
 * new entry count.  Errors: LEIDEN_EINVAL (bad IDs, self-loop, missing edge
 * or weight mismatch on deletion, duplicate deletion, unsorted rows),
 * LEIDEN_ENOMEM (result larger than cap_nnz or the context), LEIDEN_ECUDA. */
int leiden_apply_batch(leiden_ctx *ctx, const leiden_csr *g_prev, const leiden_edges *del,
                       const leiden_edges *ins, int64_t *off_out, int32_t *idx_out,
                       int32_t *w_out, int64_t cap_nnz, int64_t *nnz_out);

/* Per-call statistics of the last leiden_static / leiden_update call. */
#define LEIDEN_STATS_PASSES 32
typedef struct {
  int32_t passes;                               /* passes started */
  int32_t iters[LEIDEN_STATS_PASSES];           /* l_i of each local-moving phase */
  int64_t nv[LEIDEN_STATS_PASSES];              /* |V'| at each pass */
  int64_t nnz[LEIDEN_STATS_PASSES];             /* CSR entries of G' at each pass */
  int64_t moves[LEIDEN_STATS_PASSES];           /* local-move migrations */
  int64_t refine_moves[LEIDEN_STATS_PASSES];
  int64_t affected0;                            /* vertices unprocessed at the start */
  int64_t changed0;                             /* communities flagged changed before the first refinement */
  /* device time of the local-move decide kernels, measured with CUDA events on
   * the context stream when timing is enabled (leiden_ctx_set_timing) */
  double move_kernel_ms;
  int64_t move_kernel_launches;
  int64_t move_scanned_entries;                 /* CSR entries the decide kernels read */
  int64_t move_scanned_vertices;
  double move_bytes;                            /* algorithmic bytes of those launches */
  double total_ms;                              /* host wall time of the call */
  /* host wall time per pass: local-moving phase (with the vertex buckets),
   * refinement (with subset renumbering and the break), aggregation (with
   * renumbering and the dendrogram lookup), and the whole pass */
  double t_move_ms[LEIDEN_STATS_PASSES];
  double t_refine_ms[LEIDEN_STATS_PASSES];
  double t_agg_ms[LEIDEN_STATS_PASSES];
  double t_pass_ms[LEIDEN_STATS_PASSES];
  /* the same decide-kernel figures for the first pass alone (the first-pass
   * local-moving phase; in a profiler it is the NVTX range local_move_pass0) */
  double move0_kernel_ms;
  int64_t move0_kernel_launches;
  double move0_bytes;
  /* bit p set: pass p compared candidate scores in 128 bits, because a
   * super-vertex's K' times 2m reached 2^62 (otherwise 64 bits suffice) */
  uint32_t wide_passes;
  int64_t move0_scanned_entries;                /* CSR entries the first pass's decide kernels read */
} leiden_run_stats;

/* Copies the statistics of the last run into *out (HOST). */
int leiden_get_stats(leiden_ctx *ctx, leiden_run_stats *out);

/* Enables (1) or disables (0) CUDA-event timing of the local-move kernels. */
int leiden_ctx_set_timing(leiden_ctx *ctx, int32_t enable);

/* Allocation-free modularity.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need a
 * modularity value -- code under a memory budget that forbids new
 * allocations, plugins handed a stream but no allocator, or latency-critical
 * loops that cannot afford the device-wide synchronisation cudaMalloc and
 * cudaFree imply.  It needs no leiden_ctx and allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  Its scratch (the
 * per-community totals and accumulators) is one fixed array of about 8 MB in
 * the library's device image, which every GPU that loads the library holds
 * until the process exits; graphs above LEIDEN_NOALLOC_MAX_N vertices are
 * rejected with LEIDEN_ENOMEM.  The first call on a device looks up the
 * array's device address on that device (make it before any stream capture).
 * All calls share the array: calls that overlap on the GPU (for example on
 * two streams) race and must be serialised by the caller.  Computes Eq. 1 at
 * resolution gamma for membership (DEVICE [n], labels in [0, n)) on g, with
 * the same integer arithmetic as leiden_modularity; the work is ordered on
 * cuda_stream (cudaStream_t as void*, NULL = legacy default stream), which the
 * call synchronises before writing q_out (HOST).  The graph and the labels
 * are validated, and the verdict read on the host, before any kernel indexes
 * by them; the kernels that compute the terms test every index as well.
 * Errors: LEIDEN_EINVAL (bad gamma, malformed graph, label out of range),
 * LEIDEN_ENOMEM (n too large), LEIDEN_EOVERFLOW (nnz > 2^32 or 2m >= 2^40),
 * LEIDEN_ECUDA. */
#define LEIDEN_NOALLOC_MAX_N 1048576
int leiden_modularity_noalloc(const leiden_csr *g, const int32_t *membership, double gamma,
                              void *cuda_stream, double *q_out);

/* ---------------------------------------------------------------------------
 * Many small graphs in one persistent launch.
 *
 * leiden_batch_run takes up to max_graphs graphs at once and runs, for each,
 * the whole of Alg. leiden (every pass) inside one thread block: one kernel
 * launch for the batch, whose blocks take graphs from a device-side queue
 * (largest first) until none is left, with no host synchronisation between
 * phases.  The launch, together with the upload of the graph descriptors and
 * the download of the results, is captured once into a CUDA graph and
 * replayed for every later batch.  Same arithmetic and DET schedule as
 * leiden_static / leiden_update: for each graph the membership, modularity
 * and per-pass statistics are bit-identical to those calls.  Meant for graphs
 * small enough that one thread block per graph keeps the GPU busy; larger
 * graphs belong to a leiden_ctx.  ND, DS and DF updates recompute K^t and
 * Sigma^t from G^t and C^{t-1} (Alg. update with no auxiliary input).
 * ------------------------------------------------------------------------- */
typedef struct leiden_batch leiden_batch;

/* Creates a batch workspace bound to a stream (cudaStream_t as void*, NULL =
 * legacy default stream) for up to max_graphs graphs per run with at most
 * max_total_n vertices and max_total_nnz CSR entries summed over the run's
 * graphs (about 300 B per vertex plus 36 B per entry).  `threads` is the
 * block size of the persistent kernel (128..512, multiple of 32; 0 = 512)
 * and blocks_per_sm the number of blocks per SM it is launched with (1..4;
 * 0 = 1).  Errors: LEIDEN_EINVAL, LEIDEN_ENOMEM, LEIDEN_ECUDA. */
int leiden_batch_create(leiden_batch **out, void *cuda_stream, int32_t max_graphs, int64_t max_total_n,
                        int64_t max_total_nnz, int32_t threads, int32_t blocks_per_sm);

/* Synchronises the stream and frees the workspace.  NULL is a no-op. */
void leiden_batch_destroy(leiden_batch *b);

enum { LEIDEN_STATIC = 0 };  /* leiden_batch_item.mode for Static Leiden */

typedef struct {
  leiden_csr g;              /* the graph (G^t for updates); DEVICE pointers */
  int32_t mode;              /* LEIDEN_STATIC, LEIDEN_ND, LEIDEN_DS or LEIDEN_DF */
  int32_t reserved;          /* must be 0 */
  const int32_t *prior;      /* DEVICE [n]: C^{t-1}, labels in [0, n) (ND / DS / DF) */
  leiden_edges del, ins;     /* DEVICE: the batch that turned G^{t-1} into G^t (ND / DS / DF) */
  int32_t *membership_out;   /* DEVICE [n]: canonical labels */
} leiden_batch_item;

typedef struct {
  int32_t status;            /* LEIDEN_OK, or this graph's error (EINVAL: malformed input,
                              * EOVERFLOW: 2m >= 2^40, ECUDA: device consistency check) */
  int32_t passes;            /* passes run */
  double q;                  /* modularity (Eq. 1) at gamma of the returned membership */
  int64_t affected0, changed0;
  int32_t iters[LEIDEN_STATS_PASSES];
  int64_t nv[LEIDEN_STATS_PASSES];
  int64_t nnz[LEIDEN_STATS_PASSES];
  int64_t moves[LEIDEN_STATS_PASSES];
  int64_t refine_moves[LEIDEN_STATS_PASSES];
} leiden_batch_result;

/* Runs `count` graphs (items: HOST array) with opts (DET schedule only) and
 * writes results[k] (HOST array) for each; returns LEIDEN_OK when the batch
 * ran, even if some graphs report an error in their status.  The items'
 * device buffers must stay valid until the call returns (it synchronises the
 * stream).  Errors: LEIDEN_EINVAL (bad arguments, ASYNC schedule, a mode
 * other than the three above), LEIDEN_ENOMEM (count or the summed sizes
 * exceed the workspace), LEIDEN_ECUDA. */
int leiden_batch_run(leiden_batch *b, int32_t count, const leiden_batch_item *items, const leiden_opts *opts,
                     leiden_batch_result *results);

/* Device memory (bytes) a context's workspace holds (HOST out). */
int leiden_ctx_device_bytes(leiden_ctx *ctx, int64_t *out);

/* Device memory (bytes) a batch workspace holds (HOST out). */
int leiden_batch_device_bytes(leiden_batch *b, int64_t *out);

/* ---------------------------------------------------------------------------
 * Serving: many graphs resident on the device, continuous batching of their
 * update batches.
 *
 * A server keeps each admitted graph's CSR, membership and totals (K, Sigma)
 * resident in device memory, admitted against a byte budget that also holds
 * the server's own workspaces.  Update batches arrive at any time (from any
 * thread) and are queued per graph, applied in arrival order: G^t is built
 * from G^{t-1} and the batch (leiden_apply_batch), then C^t from C^{t-1} by
 * the configured dynamic mode (DF by default).  Worker threads take work as
 * soon as a graph and a worker are free, so requests that arrive while others
 * run join the next launch instead of waiting for a batch boundary:
 *   - graphs within the small limits go to `small_workers` workers, each of
 *     which runs every ready small request in one persistent launch
 *     (leiden_batch_run), so a new launch can start while another runs;
 *   - larger graphs go to `large_slots` workers, each with its own context and
 *     stream, so their updates overlap on the device.
 * Results are DET: each request's membership does not depend on what else
 * ran beside it.
 * ------------------------------------------------------------------------- */
typedef struct leiden_server leiden_server;

typedef struct {
  int64_t hbm_budget;        /* bytes of device memory for workspaces and resident graphs */
  int32_t large_slots;       /* concurrent workers for large graphs (>= 1) */
  int32_t small_max_graphs;  /* graphs per persistent launch (>= 1) */
  int64_t large_max_n;       /* largest graph a large worker's context holds */
  int64_t large_max_nnz;
  int64_t small_max_n;       /* a graph with n <= small_max_n and capacity <= small_max_nnz */
  int64_t small_max_nnz;     /*   CSR entries runs on the persistent path */
  int64_t small_batch_n;     /* vertices / entries summed over one persistent launch */
  int64_t small_batch_nnz;
  double growth;             /* spare CSR capacity of a resident graph, as a fraction of its nnz */
  int32_t mode;              /* LEIDEN_DF (default when 0), LEIDEN_DS or LEIDEN_ND */
  int32_t autotune_trials;   /* > 0: leiden_autotune each large graph at admission with this many
                              * candidate tier tables and use its table for the graph's runs */
  int32_t small_workers;     /* workers for small graphs, each with its own persistent launch in
                              * flight (>= 1; 0 = 2) */
  int32_t min_persistent;    /* fewer ready small graphs than this run one by one on the worker's
                              * context (all SMs on one graph) instead of one persistent launch
                              * (one block per graph); 0 = 8 */
  leiden_opts opts;          /* DET schedule */
} leiden_server_config;

/* Fills a default configuration (HOST): 16 GB budget, 2 large slots, 2
 * small-graph workers, 64 graphs per persistent launch, small graphs up to
 * 2^16 vertices / 2^18 entries, 25% growth, DF, default options. */
void leiden_server_config_default(leiden_server_config *cfg);

/* Creates a server on the current device and starts its workers.  Errors:
 * LEIDEN_EINVAL, LEIDEN_ENOMEM (the workspaces exceed the budget), ECUDA. */
int leiden_server_create(leiden_server **out, const leiden_server_config *cfg);

/* Finishes the queued work, stops the workers, frees everything. */
void leiden_server_destroy(leiden_server *s);

/* Admits a graph (HOST CSR, copied to the device) if its footprint -- two
 * CSR buffers of nnz * (1 + growth) entries, membership and totals -- fits
 * the remaining budget, and queues its Static Leiden; *graph_id receives its
 * handle and *request_id (may be NULL) the Static request.  Errors:
 * LEIDEN_EINVAL (malformed sizes), LEIDEN_ENOMEM (over budget or too large
 * for every worker). */
int leiden_server_admit(leiden_server *s, int64_t n, int64_t nnz, const int64_t *off, const int32_t *idx,
                        const int32_t *w, int32_t *graph_id, int64_t *request_id);

/* Queues an update batch (HOST arrays in del / ins, copied) for a graph;
 * *request_id receives its handle.  Errors: LEIDEN_EINVAL (unknown graph,
 * bad sizes). */
int leiden_server_submit(leiden_server *s, int32_t graph_id, const leiden_edges *del, const leiden_edges *ins,
                         int64_t *request_id);

typedef struct {
  int32_t status;            /* LEIDEN_OK or the request's error */
  int32_t graph;
  int32_t path;              /* 0: persistent many-graph launch, 1: large-graph worker,
                              * 2: small-graph worker on its own context (few graphs ready) */
  int32_t launch_graphs;     /* graphs in the same persistent launch (path 0) */
  double q;                  /* modularity of the new membership */
  double queue_ms;           /* submission to start of its work */
  double latency_ms;         /* submission to result ready */
  int64_t n, nnz;            /* of the graph after the request */
} leiden_request_info;

/* Waits up to timeout_ms (< 0: forever) for a request; LEIDEN_ETIMEOUT if it
 * is not done by then.  *out (HOST) receives its record, after which the
 * request is forgotten: each request is waited on once (a second wait gets
 * LEIDEN_EINVAL). */
int leiden_server_wait(leiden_server *s, int64_t request_id, double timeout_ms, leiden_request_info *out);

/* Copies a graph's current membership (n labels) into host_out, after
 * waiting for its queued requests. */
int leiden_server_membership(leiden_server *s, int32_t graph_id, int32_t *host_out, int64_t n);

/* Waits for a graph's queued requests, then frees its device memory. */
int leiden_server_evict(leiden_server *s, int32_t graph_id);

typedef struct {
  int64_t resident_graphs, resident_bytes, workspace_bytes, budget;
  int64_t completed, failed, small_launches, small_graphs_launched, large_runs;
} leiden_server_stats;

int leiden_server_get_stats(leiden_server *s, leiden_server_stats *out);

/* Number of CUDA kernels this library has enqueued in this process so far,
 * over all contexts, devices and threads (a relaxed atomic counter; every
 * replay of a captured CUDA graph counts the kernels it runs).  Callers
 * difference two readings to count the launches of a region. */
uint64_t leiden_kernel_launches(void);

/* Degree tiers of the local-moving and refinement kernels.  A vertex whose
 * CSR row has d entries is processed by the first tier with d <= max_degree
 * (vertices with d = 0 are never processed).  A GROUP tier gives each vertex
 * `lanes` lanes of a warp and a shared-memory hashtable of 2^log2_slots
 * slots; a BLOCK tier gives it a block of `threads` threads and a
 * shared-memory table of 2^log2_slots slots; the HUB tier (always the last,
 * max_degree unbounded) spreads each row over many blocks with tables in
 * global scratch.  The tier table changes only the kernel shapes, never the
 * result: every vertex takes the same decision whichever tier processes it.
 * The default table is the one leiden_tiers_default returns; leiden_autotune
 * picks one per graph. */
#define LEIDEN_MAX_TIERS 11
enum { LEIDEN_TIER_GROUP = 1, LEIDEN_TIER_BLOCK = 2, LEIDEN_TIER_HUB = 3 };
typedef struct {
  int32_t kind;        /* LEIDEN_TIER_GROUP, LEIDEN_TIER_BLOCK or LEIDEN_TIER_HUB */
  int32_t lanes;       /* GROUP: lanes per vertex, 1, 4, 8, 16 or 32; otherwise 0 */
  int32_t log2_slots;  /* GROUP: (lanes, log2_slots) in (1,2) (1,3) (4,3) (4,4) (8,4) (8,5) (16,5)
                        * (16,6) (32,6..10); with 1 lane the row is held in 2^log2_slots
                        * registers (max_degree <= 2^log2_slots) instead of a table;
                        * BLOCK: 6..14; HUB: 0 */
  int32_t threads;     /* GROUP: 32..256, BLOCK: 64..1024, multiples of 32; HUB: 0 */
  int64_t max_degree;  /* inclusive upper end of the degree range; HUB: ignored */
} leiden_tier;
typedef struct {
  int32_t count;       /* tiers in use, 1..LEIDEN_MAX_TIERS; the last one is the HUB tier */
  int32_t reserved;    /* must be 0 */
  leiden_tier tier[LEIDEN_MAX_TIERS];
} leiden_tier_table;

/* Fills the default tier table (HOST). */
void leiden_tiers_default(leiden_tier_table *out);

/* Checks a tier table (HOST, no GPU needed): kinds and shapes from the lists
 * above, max_degree increasing, 2^log2_slots >= 2 * max_degree for GROUP and
 * BLOCK tiers (a table never fills past half; >= max_degree for a one-lane
 * GROUP tier), shared memory within 227 KB per block, exactly one HUB tier,
 * last.  Returns LEIDEN_OK or LEIDEN_EINVAL. */
int leiden_tiers_validate(const leiden_tier_table *t);

/* Sets the context's tier table (HOST; NULL restores the default) for its
 * following runs; LEIDEN_EINVAL if leiden_tiers_validate rejects it (the
 * context keeps its table). */
int leiden_ctx_set_tiers(leiden_ctx *ctx, const leiden_tier_table *t);

/* Aggregation policy (Alg. leidenag) of the context's following runs.
 * LEIDEN_AGG_TIERED (the default) gives each community a kernel shape sized
 * to its total degree -- a warp with a shared-memory table, a block, or, for
 * giant communities, fixed-size buckets spread over many blocks -- the GPU
 * form of the paper's Optimized Aggregation (Sec. 4.4: small work units so
 * that one large unrefined community does not hold up a worker).
 * LEIDEN_AGG_UNIFORM sends every community through the bucketed path, one
 * method for all sizes, for the ablation of Sec. 4.2-4.4.  The result is the
 * same either way.  Errors: LEIDEN_EINVAL. */
enum { LEIDEN_AGG_TIERED = 0, LEIDEN_AGG_UNIFORM = 1 };
int leiden_ctx_set_agg_policy(leiden_ctx *ctx, int32_t policy);

/* Copies the context's tier table into *out (HOST). */
int leiden_ctx_get_tiers(leiden_ctx *ctx, leiden_tier_table *out);

/* Autotuner of the tier table.  Times leiden_static on g with opts (the
 * context's stream, CUDA events) for each of up to max_trials candidate
 * tables -- degree thresholds of the group, block and hub tiers, hashtable
 * load factors and block shapes drawn from a fixed candidate list ordered by
 * expected benefit -- taking the median of `repeats` runs each (>= 1), and
 * sets the fastest on the context.  best_out (HOST, may be NULL) receives
 * that table and best_ms (HOST, may be NULL) its median time.  The partition
 * is the same for every candidate (DET); membership is not returned.  Errors:
 * those of leiden_static. */
int leiden_autotune(leiden_ctx *ctx, const leiden_csr *g, const leiden_opts *opts, int32_t max_trials,
                    int32_t repeats, leiden_tier_table *best_out, double *best_ms);

/* Detail of the context's last failure (a CUDA error name and message, or a
 * device consistency check), empty if none; owned by the context and valid
 * until its next call. */
const char *leiden_ctx_last_error(leiden_ctx *ctx);

/* Human-readable name of an error code (static storage). */
const char *leiden_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
