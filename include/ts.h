/*
 * ts.h -- C ABI of libts_gb300, a GB300 (sm_103a) distance threshold search over historical
 * continuous trajectories, after Gowanlock & Casanova, "Towards Efficient Indexing of
 * Spatiotemporal Trajectories on the GPU for Distance Threshold Similarity Searches".
 *
 * Problem (Sec. 3.1): a database D of 4-D line segments (x, y, z, t start point to end point;
 * linear motion in between) and a set Q of query segments. For a distance d and a query interval
 * [t_start, t_end] the search returns every (q, l) pair whose common time window, clipped to the
 * interval, has positive length and contains instants at which the two moving points are within
 * d of each other, together with the sub-interval [t_in, t_out] of those instants (a convex
 * quadratic's non-positive set, so one interval per pair).
 *
 * D and its index are built once and stay resident on the GPU; they are queried many times
 * (Sec. 3.1, platform). Three indexes prune the candidates (Sec. 4.1 spatial grid, Sec. 4.2
 * temporal bins, Sec. 4.3 spatiotemporal subbins); all return the same pair set as the plain
 * all-pairs search (TS_INDEX_BRUTE).
 *
 * Conventions of every call:
 *  - Status codes: every call returns ts_status; nothing throws across this boundary. On error a
 *    thread-local message is available from ts_last_error().
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Work
 *    is stream ordered.
 *  - Pointers: ts_segments arrays are device pointers unless on_host = 1; they stay owned by the
 *    caller and are only read.
 *  - Precision: coordinates, times, d and result times are IEEE FP64.
 *  - Handles: ts_index and ts_result are opaque, owned by the library and released with
 *    ts_free(). An index is immutable after ts_build_index() returns and can be searched from
 *    several host threads and streams at once.
 *  - Determinism: for a given index, query set and parameters the rows, their order and every
 *    bit of t_in / t_out are the same from run to run.
 */
#ifndef TS_GB300_H
#define TS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ts_status {
    TS_OK = 0,
    TS_ERR_INVALID_ARG = 1, /* bad argument or input value (NaN/Inf, t_end <= t_start, d <= 0) */
    TS_ERR_OOM = 2,         /* device or host allocation failed */
    TS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error string) */
    TS_ERR_CAPACITY = 4,    /* result count above the caller's max_results (count still given) */
    TS_ERR_TIMEOUT = 5,     /* a bounded device-side or host-side wait ran out */
    TS_ERR_CANCELLED = 6,   /* the request was cancelled (server) */
    TS_ERR_INTERNAL = 7     /* an internal consistency check failed */
} ts_status;

typedef enum ts_index_kind {
    TS_INDEX_BRUTE = 0,          /* no pruning: every query against every entry (reference mode) */
    TS_INDEX_SPATIAL = 1,        /* flatly structured grid, Sec. 4.1 (GPUSpatial) */
    TS_INDEX_TEMPORAL = 2,       /* temporal bins, Sec. 4.2 (GPUTemporal) */
    TS_INDEX_SPATIOTEMPORAL = 3  /* temporal bins split into spatial subbins, Sec. 4.3 */
} ts_index_kind;

/* A set of line segments in structure-of-arrays FP64 form (Sec. 3.1): segment i goes from
 * (x0[i], y0[i], z0[i]) at time t0[i] to (x1[i], y1[i], z1[i]) at time t1[i], t1[i] > t0[i]. */
typedef struct ts_segments {
    const double *x0, *y0, *z0, *t0;
    const double *x1, *y1, *z1, *t1;
    uint64_t n;       /* number of segments; at most 2^31 - 1 */
    int32_t on_host;  /* 0: device pointers; 1: host pointers, copied to the device by the call */
    int32_t reserved;
} ts_segments;

/* Index parameters; 0 selects the library's default for that field. */
typedef struct ts_index_params {
    int32_t kind;        /* ts_index_kind */
    uint32_t t_bins;     /* m: temporal bins (Sec. 4.2); used by TEMPORAL and SPATIOTEMPORAL */
    uint32_t sub_bins;   /* v: subbins per dimension (Sec. 4.3), lowered per dimension so that a
                            subbin is at least as wide as the longest entry in that dimension */
    uint32_t grid_cells; /* cells per dimension of the spatial grid (Sec. 4.1), at most 512 */
} ts_index_params;

/* Search parameters. */
typedef struct ts_query_params {
    double d;            /* distance threshold, finite and > 0 */
    double t_start;      /* query interval [t_start, t_end] (Sec. 1); t_start <= t_end */
    double t_end;
    uint64_t max_results; /* 0 = unlimited; else more rows -> TS_ERR_CAPACITY (paper's result
                             buffer and incremental processing, Sec. 5.2) */
} ts_query_params;

/* Counters of one search (all exact, counted on the device). */
typedef struct ts_search_stats {
    uint64_t n_queries;   /* query segments passed in */
    uint64_t n_qsegs;     /* query segments with a positive-length overlap with [t_start, t_end] */
    uint64_t n_tests;     /* candidate (query, entry) pairs the index produced and the pair
                             kernel evaluated */
    uint64_t n_exact;     /* candidates that passed the conservative FP32 filter and were
                             decided by the FP64 test */
    uint64_t n_hits;      /* result rows */
    uint64_t n_tiles;     /* work tiles (query group x candidate range) */
    uint64_t n_groups;    /* query groups (up to 32 queries sharing a candidate range) */
    uint64_t n_subbin;    /* queries served from a subbin range (spatiotemporal index) */
    double ms_count_pass; /* device time of the pair kernel's count pass (CUDA events) */
    double ms_write_pass; /* device time of the pair kernel's write pass (CUDA events) */
    /* how the pair kernel's count pass swept the candidates (diagnostics): */
    uint64_t n_chunks;    /* (tile, chunk of 64 entries) pairs swept */
    uint64_t n_dense;     /* chunks swept by the two-axis bitmask (more than 8 members meet them) */
    uint64_t n_sparse;    /* (member, chunk) visits of the per-member path (few members meet) */
    uint64_t n_stage2;    /* bitmask survivors given the full FP32 box and gap filters */
} ts_search_stats;

/* Read-only description of a built index. */
typedef struct ts_index_info {
    int32_t kind;
    uint32_t t_bins;        /* m actually used */
    uint32_t sub_bins[3];   /* v actually used per dimension (x, y, z) */
    uint32_t grid_cells;    /* cells per dimension actually used */
    uint64_t n;             /* entry segments */
    uint64_t st_len[3];     /* length of the X, Y, Z id arrays (Sec. 4.3) */
    uint64_t grid_len;      /* length of the grid lookup array A (Sec. 4.1) */
    uint64_t device_bytes;  /* device memory held by the index */
    double t_min, t_max, bin_width;
    double sub_lo[3], sub_w[3];
    double grid_lo[3], grid_w[3];
} ts_index_info;

typedef struct ts_index ts_index;
typedef struct ts_result ts_result;

/*
 * Build the index of database `db` (Sec. 4.1-4.3). The database is validated (finite values,
 * t1 > t0; else TS_ERR_INVALID_ARG), sorted by start time (Sec. 4.2), given velocities, and
 * binned; the segments are copied, so the caller may release db's arrays once the call returns.
 * The call synchronises `stream` (index building is offline work, Sec. 5.2). On success *out
 * owns the index (release with ts_free).
 */
ts_status ts_build_index(const ts_segments *db, const ts_index_params *params, void *stream,
                         ts_index **out);

/* Describe a built index. */
ts_status ts_index_get_info(const ts_index *idx, ts_index_info *info);

/* Fields exported by ts_index_export (for inspection and tests). `dim` selects x/y/z where noted. */
typedef enum ts_index_field {
    TS_FIELD_PERM = 0,       /* uint32[n]: sorted position -> caller's entry index (Sec. 4.2) */
    TS_FIELD_BIN_START = 1,  /* double[m]: B_j^start */
    TS_FIELD_BIN_END = 2,    /* double[m]: B_j^end */
    TS_FIELD_BIN_OFF = 3,    /* uint32[m+1]: first entry of bin j (B_j^first), last = next - 1 */
    TS_FIELD_ST_IDS = 4,     /* uint32[st_len[dim]]: X, Y or Z id array (sorted positions) */
    TS_FIELD_ST_OFF = 5,     /* uint32[v*m+1]: subbin (i, j) range starts at off[j*m + i] */
    TS_FIELD_GRID_A = 6,     /* uint32[grid_len]: lookup array A (sorted positions) */
    TS_FIELD_GRID_OFF = 7    /* uint32[g^3+1]: cell h range starts at off[h] */
} ts_index_field;

/* Copy one internal array of the index to host memory `dst` of `capacity` bytes. *size receives
 * the array's byte size; TS_ERR_CAPACITY (nothing copied) when capacity is too small. */
ts_status ts_index_export(const ts_index *idx, int32_t field, int32_t dim, void *dst,
                          uint64_t capacity, uint64_t *size);

/*
 * Per-query candidate schedule (Sec. 4.2 schedule S, Sec. 4.3 schedule with array selector):
 * for every query segment, in the caller's order, sel = 0/1/2 for a range of the X/Y/Z id array,
 * 3 for a range of the time-sorted entries; [lo, hi) is the half-open range. Queries whose
 * clipped window is empty get sel = 3, lo = hi = 0. For TS_INDEX_BRUTE the range is [0, n); for
 * TS_INDEX_SPATIAL, sel = 4 and lo/hi hold the number of raw and duplicate-free candidates.
 * sel, lo, hi are host arrays of q->n elements. Synchronises `stream`.
 */
ts_status ts_schedule(const ts_index *idx, const ts_segments *q, const ts_query_params *qp,
                      void *stream, int32_t *sel, uint64_t *lo, uint64_t *hi);

/*
 * Search the index with the query segments `q` (Alg. 1-3 of the paper, re-designed: count pass,
 * exclusive scan, write pass, so the output is exact-size and deterministic). Rows are grouped by
 * work tile in a fixed tile order; sort by (q_idx, e_idx) for a canonical order. q_idx is the
 * caller's query index, e_idx the caller's database index. The call synchronises `stream` once
 * (to size the result). On TS_ERR_CAPACITY *out still receives a result whose count is the exact
 * number of rows and whose row arrays are empty, so the caller can split Q and retry.
 */
ts_status ts_search(const ts_index *idx, const ts_segments *q, const ts_query_params *qp,
                    void *stream, ts_result **out);

/*
 * Stationary-point search (the fixed-point queries of Sec. 1, e.g. every star that comes within d
 * of a supernova's position while its radiation passes): every database segment within d of one
 * of n fixed points (x[i], y[i], z[i]) at some instant of [qp->t_start, qp->t_end]. Each point is
 * searched as a query segment that stays at its position over the whole interval (zero spatial
 * length, a valid segment of Sec. 3.1), so the pair test and its interval are the general ones.
 * x, y, z: n doubles each, in host memory when on_host is non-zero, else in device memory (read
 * on `stream`). The interval must have positive length (TS_ERR_INVALID_ARG otherwise). q_idx in
 * the result is the point's index; results, capacity and errors are as for ts_search.
 */
ts_status ts_search_points(const ts_index *idx, const double *x, const double *y, const double *z,
                           uint64_t n, int32_t on_host, const ts_query_params *qp, void *stream,
                           ts_result **out);

/* Number of rows of a result. */
uint64_t ts_result_count(const ts_result *r);

/* Device pointers to the result rows (structure of arrays, ts_result_count elements each, owned
 * by the result). NULL pointers are allowed for fields the caller does not need. */
ts_status ts_result_arrays(const ts_result *r, const uint32_t **q_idx, const uint32_t **e_idx,
                           const double **t_in, const double **t_out);

/* Counters of the search that produced `r`. */
ts_status ts_result_stats(const ts_result *r, ts_search_stats *stats);

/* Copy the rows to host arrays of at least ts_result_count elements (NULL = skip the field).
 * Synchronises `stream`. */
ts_status ts_result_copy_to_host(const ts_result *r, uint32_t *q_idx, uint32_t *e_idx,
                                 double *t_in, double *t_out, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Batched search. Many requests (each a query set with its own d and interval) run through one
 * pipeline: one query preparation launch, one sort of all candidate ranges, one persistent pair
 * kernel per pass pulling work tiles of all requests from a device queue. The paper searches one
 * query set per kernel invocation (Sec. 4); batching is this library's extension for serving.
 * ------------------------------------------------------------------------------------------- */

/* One-shot batch: nreq requests qs[r] with parameters qps[r]; outs[r] receives request r's result
 * (q_idx relative to qs[r]); the results share one device allocation that is released when the
 * last of them is freed. Synchronises `stream`. On TS_ERR_CAPACITY (some request over its
 * max_results) every outs[r] still carries its exact count and no rows. */
ts_status ts_search_batch(const ts_index *idx, uint32_t nreq, const ts_segments *qs,
                          const ts_query_params *qps, void *stream, ts_result **outs);

/* Reusable batch plan with fixed capacities; every run is free of host synchronisation and, with
 * use_graph, is captured once in a CUDA graph and replayed. */
typedef struct ts_batch_params {
    uint32_t max_requests;  /* requests per run, < 2^24 */
    uint32_t tile_records;  /* candidate records per work tile, multiple of 64, <= 2048 (0 = 256) */
    uint64_t max_queries;   /* query segments per run, all requests together */
    uint64_t max_rows;      /* result rows per run, all requests together */
    uint64_t max_units;     /* candidate ranges per run (0 = derived) */
    uint64_t max_tiles;     /* work tiles per run (0 = derived) */
    int32_t use_graph;      /* 1: capture the run in a CUDA graph once, then replay it */
    int32_t pair_blocks;    /* blocks of the persistent pair kernel (0 = all resident) */
    uint64_t scratch_rows;  /* hits the count pass keeps (32 B each) and places after the scan;
                               a run with more hits sweeps its tiles a second time to write them
                               (0 = max_rows) */
} ts_batch_params;

typedef struct ts_batch ts_batch;

/* Outcome of the last run of a plan. */
typedef struct ts_batch_status {
    uint64_t rows;          /* result rows of the run (exact, also when over capacity) */
    uint32_t nreq;
    int32_t overflow;       /* 1: a capacity was exceeded; no rows were written */
    ts_search_stats stats;  /* totals over all requests of the run */
} ts_batch_status;

/* Create a plan for `idx` (device memory for all capacities is allocated here, once). */
ts_status ts_batch_create(const ts_index *idx, const ts_batch_params *params, void *stream,
                          ts_batch **out);

/* Enqueue one run of nreq <= max_requests requests on `stream` (the plan's stream when NULL).
 * Query columns may be device pointers or host pointers (on_host = 1). Host columns in pinned
 * (page-locked) memory are read by the device in place and must stay valid until ts_batch_wait;
 * other host columns are copied into the plan's pinned staging by this call. Returns without
 * waiting for the device. The plan's previous run must have been waited for. */
ts_status ts_batch_run(ts_batch *b, uint32_t nreq, const ts_segments *qs,
                       const ts_query_params *qps, void *stream);

/* Wait for the last run (only for it and the work enqueued before it on its stream: plans that
 * share a stream, run one after another, are waited for one by one) and report its outcome. */
ts_status ts_batch_wait(ts_batch *b, ts_batch_status *status);

/* Rows of request r of the last run: [first, first + count) of the plan's row arrays, whose
 * device pointers ts_batch_rows returns (valid until the next run). q_idx is relative to the
 * request's query set. */
ts_status ts_batch_request_rows(const ts_batch *b, uint32_t r, uint64_t *first, uint64_t *count);
ts_status ts_batch_rows(const ts_batch *b, const uint32_t **q_idx, const uint32_t **e_idx,
                        const double **t_in, const double **t_out);

/* Copy rows [first, first + count) of the last run to host arrays (NULL = skip a field). The
 * copies run on the plan's own stream after the last run and are waited for; work enqueued after
 * that run on a stream the plan shares keeps running meanwhile. */
ts_status ts_batch_copy_rows(const ts_batch *b, uint64_t first, uint64_t count, uint32_t *q_idx,
                             uint32_t *e_idx, double *t_in, double *t_out);

/* ---------------------------------------------------------------------------------------------
 * Served search: a request loop on a resident index ("D is stored once and queried multiple
 * times", Sec. 3.1). Requests are submitted from any host thread; a loop thread admits them into
 * batches while a batch's query and row capacity allow, runs up to max_inflight batches at once
 * on their own streams (a batch is formed while another runs), splits a batch whose rows
 * overflow, and hands every request its own result. Every wait is bounded.
 * ------------------------------------------------------------------------------------------- */
typedef struct ts_server_params {
    uint32_t max_inflight;        /* batches on the device at once (>= 1; 2 overlaps batches) */
    uint32_t max_batch_requests;  /* requests per batch */
    uint64_t max_batch_queries;   /* query segments per batch (admission capacity) */
    uint64_t max_batch_rows;      /* result rows of a batch: its count pass sizes the rows
                                     exactly; a batch with more is split, a lone request with
                                     more ends with TS_ERR_CAPACITY */
    uint32_t tile_records;        /* as in ts_batch_params */
    int32_t use_graph;            /* replay each batch plan as a CUDA graph */
    uint32_t linger_us;           /* how long a partly filled batch waits for more requests */
    uint32_t admit_wait_ms;       /* how long a counted batch waits for room in the memory budget
                                     before it is admitted beyond the budget, if the device has
                                     the memory (0 = 1000 ms); results that completed but were
                                     not yet collected hold budget too, so an unbounded wait
                                     could wait on a client that waits on this batch */
    uint64_t scratch_rows;        /* hits a batch's count pass keeps for placement (0 = derived
                                     from the budget: an eighth of it per plan, at 32 B per
                                     hit); the tiles of hits beyond it are swept a second time */
    uint64_t mem_budget_bytes;    /* device memory the server may hold: its plans (work buffers
                                     and scratch) and the rows of results not yet released
                                     (0 = three quarters of the free device memory at creation).
                                     A batch whose rows do not fit beside the rows still held
                                     waits (its plan idle) until results are released, for at
                                     most admit_wait_ms; one whose rows alone exceed the budget
                                     is split */
} ts_server_params;

typedef struct ts_server ts_server;

/* Host-clock timestamps of a served request, in microseconds since the server started. */
typedef struct ts_request_timing {
    double submit_us, start_us, done_us;
    uint32_t batch_requests;  /* requests in the batch that served it */
    uint32_t requeued;        /* times its batch went back to the queue (split, plan growth) */
} ts_request_timing;

ts_status ts_server_create(const ts_index *idx, const ts_server_params *params,
                           ts_server **out);

/* Submit a request: its query segments (host or device arrays; copied before the call returns)
 * and parameters. *ticket identifies it in ts_server_wait. */
ts_status ts_server_submit(ts_server *srv, const ts_segments *q, const ts_query_params *qp,
                           uint64_t *ticket);

/* Wait up to timeout_ms for a request. On success *out receives its result (device rows, release
 * with ts_free) and *timing its timestamps (may be NULL). TS_ERR_TIMEOUT leaves the request in
 * place; any other status is the request's own outcome and ends its ticket. */
ts_status ts_server_wait(ts_server *srv, uint64_t ticket, uint32_t timeout_ms, ts_result **out,
                         ts_request_timing *timing);

/* The server's device-memory accounting: its budget (mem_budget_bytes, or the one derived at
 * creation), the bytes its batch plans hold, and the bytes of result rows not yet released (any
 * pointer may be NULL). A service of the request loop; the paper has no counterpart. */
ts_status ts_server_info(ts_server *srv, uint64_t *budget_bytes, uint64_t *plan_bytes,
                         uint64_t *held_bytes);

/* Cancel a request that has not started; TS_ERR_INVALID_ARG when it already started or ended. */
ts_status ts_server_cancel(ts_server *srv, uint64_t ticket);

/* Stop the loop (waits for in-flight batches) and release the server. Requests still queued end
 * with TS_ERR_CANCELLED. */
void ts_server_destroy(ts_server *srv);

/* Release a ts_index, ts_result or ts_batch (NULL is a no-op). Waits for the device work of the
 * handle. */
void ts_free(void *handle);

/* Message of the last failed call on this host thread ("" if none). */
const char *ts_last_error(void);

/*
 * All-pairs search that allocates nothing (the paper has no counterpart; this is a service of this
 * library). It is meant for callers that cannot call cudaMalloc: code embedded in an application
 * that owns all device memory through its own allocator or a fixed budget, where a library-side
 * cudaMalloc would escape that accounting or fail, and latency-bound request paths where
 * cudaMalloc/cudaFree, which may synchronise the device, are not acceptable.
 *
 * Same result set and FP64 test as ts_search on a TS_INDEX_BRUTE index (every query segment
 * against every database segment, no index). db and q must be device arrays (on_host = 0); the
 * caller provides the output arrays q_idx, e_idx, t_in, t_out of `capacity` rows (device memory).
 * *count receives the number of rows; when it exceeds `capacity` the call returns
 * TS_ERR_CAPACITY and writes no rows. Rows are in tile order (32 query segments x 1024 database
 * segments); sort by (q_idx, e_idx) for a canonical order. The call synchronises `stream`.
 *
 * Working memory: a fixed TS_NOALLOC_SCRATCH_BYTES (32 MiB) device array that is part of the
 * library image; every GPU that loads the library holds it until the process exits. Problems
 * needing more than TS_NOALLOC_MAX_TILES tiles, i.e. ceil(q->n / 32) * ceil(db->n / 1024) >
 * 2,500,000, are rejected with TS_ERR_CAPACITY before any device work. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current, so make
 * that first call before any stream capture. All calls share the one array and it keeps the last
 * call's contents: calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. The call makes no cudaMalloc, cudaFree or other allocating
 * call.
 */
#define TS_NOALLOC_SCRATCH_BYTES (32ull << 20)
#define TS_NOALLOC_MAX_TILES 2500000ull
ts_status ts_search_brute_noalloc(const ts_segments *db, const ts_segments *q,
                                  const ts_query_params *qp, uint32_t *q_idx, uint32_t *e_idx,
                                  double *t_in, double *t_out, uint64_t capacity, uint64_t *count,
                                  void *stream);

/* Number of kernels this library has launched in this process so far (all streams, all
 * devices); the difference across a region counts the launches inside it. */
uint64_t ts_kernel_launches(void);

/* Measured arithmetic peaks of the current device, in TFLOP/s (an FMA counts two flops): FP32
 * and FP64 fused multiply-add loops over every SM, timed with CUDA events (best of 3 after a
 * warm-up; ~0.3 s in total). These are the denominators of the pair kernel's roofline (its filter
 * runs on the FP32 pipe, its exact test on the FP64 pipe); the paper has no counterpart. */
ts_status ts_measure_alu_peaks(double *fp32_tflops, double *fp64_tflops);

/* The exact test's reciprocal and square root beside the CUDA runtime's, for n values x (host
 * arrays of n doubles each; the call allocates a small device buffer and synchronises the device).
 * The interval of a hit (the roots s/a and c/s of Sec. 3.1's distance quadratic) uses a hardware
 * reciprocal or reciprocal-square-root estimate refined by one Newton-Raphson step (about 2^-40
 * relative error, against the search's 1e-9 interval tolerance); this call
 * evaluates those refinements on the device (rcp_est, sqrt_est; NaN outside their range,
 * 2^-1000 <= |x| < 2^1000) and the correctly rounded 1/x and sqrt(x) (rcp_ref, sqrt_ref) so a
 * test can bound their difference. A diagnostic; the paper has no counterpart. */
ts_status ts_eval_refined_estimates(const double *x, uint64_t n, double *rcp_est,
                                    double *sqrt_est, double *rcp_ref, double *sqrt_ref);

/* Test hook of the device-side timeout path (the paper has no counterpart). Every wait of the
 * pair kernel on a bulk copy is bounded (2 s of the GPU's global timer); when one runs out, the
 * kernel records TS_ERR_TIMEOUT in the search's status word, waits (bounded) for its own copies
 * still in flight and returns, so the context stays usable. After this call, the count pass of
 * the next plain search (ts_search or ts_search_points, on any thread) has one warp wait limit_ns
 * nanoseconds (at most 1e9) on a barrier phase that never completes, then take that path: that
 * search returns TS_ERR_TIMEOUT. Batch plans and the served loop are not affected. */
ts_status ts_debug_inject_stall(uint64_t limit_ns);

/* Library version string. */
const char *ts_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TS_GB300_H */
