// ts_search.cuh -- the search pipeline shared by the plain, batched and served paths.
//
// A batch holds R requests (query set, d, [t_start, t_end]); the plain search is R = 1.
//   1. query preparation (one thread per query segment): validation, clipped window, FP64 query
//      record, FP32 boxes, and the query's candidate units -- (array, range) pairs from the
//      index's schedule (Sec. 4.2 / 4.3), or one unit per z-run of grid cells (Sec. 4.1);
//   2. units sorted by (request, array, range start);
//   3. groups of up to 32 consecutive units of one request; the union of their ranges is merged
//      into disjoint segments, cut into tiles of PK_TILE records;
//   4. pair kernel, count pass: per tile the number of hits;
//   5. exclusive scan of the tile counts (row offsets; a request's rows are contiguous);
//   6. pair kernel, write pass: rows at their offsets.
#pragma once

#include "ts_index.cuh"

namespace ts {

constexpr int PK_WARPS = 8;
constexpr int PK_THREADS = PK_WARPS * 32;
constexpr int PK_CH = 64;      // records per bulk-copy stage (2 KB): 2 per lane
constexpr int PK_STAGES = 2;   // chunk stages per warp (copies in flight while one is swept)
constexpr int PK_QUEUE = 64;   // exact-test queue per warp (drained at 32)
constexpr uint32_t PK_PLIST = 128;  // box-test survivors of a chunk awaiting the gap bound
constexpr uint32_t PK_MAX_TILES = (1u << 29) - 1;  // tile index bits of a queued candidate
constexpr int PK_SPARSE = 8;  // chunks met by at most this many members: per-member sweep
constexpr int PK_TILE = 256;   // records per tile (multiple of PK_CH)
constexpr int GROUP = 32;      // units per group
constexpr int PK_MIN_BLOCKS = 2;  // resident pair-kernel blocks per SM the register budget targets

// run header words: valid units, groups, tiles (low, high), unit slots holding a sort key
enum { HDR_U = 0, HDR_G = 1, HDR_T_LO = 2, HDR_T_HI = 3, HDR_NU = 4, HDR_N = 5 };

// One request of a batch (device memory).
struct ReqDesc {
    double d, dd, t_start, t_end;
    uint32_t q_first, q_count;  // its queries in the batch's concatenated query arrays
    float d_up, d2u;            // FP32 upper bounds of d and of d^2 (with slack)
    float d_dn, pad;            // FP32 lower bound of d
    const double *cols[8];      // batched runs: the request's query columns (device-readable)
};

// A group member as the pair kernel reads it (one bulk copy per tile): the query's d-expanded
// FP32 box (with its clipped window), the unit's own range in its array, the query index in the
// batch and the array.
struct __align__(16) MemberRec {
    float4 ea, eb;
    uint32_t lo, hi, qi, sel;
};
static_assert(sizeof(MemberRec) == 48, "MemberRec is 48 bytes");

// Device buffers of one pipeline run (pointers; ownership outside).
struct PipeBufs {
    // per query
    QueryD *qd;
    float4 *qf;          // 2 per query: d-expanded box lo (+ window start), hi (+ window end)
    uint32_t *qreq;      // request of every query
    uint32_t *qcell;     // grid only: 6 x 10-bit cell box packed into two u32 per query
    uint32_t *qnu;       // grid only: units per query
    uint32_t *quoff;     // grid only: exclusive scan of qnu (nq + 1)
    // per unit (unit id order)
    uint32_t *u_q, *u_lo, *u_hi, *u_sel;
    uint64_t *keys;
    uint32_t *vals;      // sorted unit ids after the sort
    // per request
    uint32_t *req_units, *ustart, *req_groups, *gstart;  // R, R+1, R, R+1
    // groups
    uint32_t *g_first, *g_count, *g_nseg;
    MemberRec *gmem;      // GROUP per group, in the group's (array, start) order
    float4 *ghdr;         // per group: its request's d_dn, d2u, q_first (bits), 0
    uint32_t *seg_lo, *seg_hi, *seg_sel, *seg_t0;  // GROUP per group
    uint32_t *ntiles;
    uint64_t *tile_base;  // groups + 1
    // tiles and rows
    uint4 *tdesc;         // per tile: {group, s0, s1, sel | (members - 1) << 3 | request << 8}
    uint32_t *tile_hits;
    uint64_t *tile_off;   // tiles + 1
    uint32_t *out_q, *out_e;
    double *out_tin, *out_tout;
    // hits found by the count pass (tile, rank in the tile, row), placed after the scan
    uint32_t *s_tile, *s_rank, *s_q, *s_e;
    double *s_tin, *s_tout;
    // control
    uint32_t *hdr;
    unsigned long long *stats;
    uint32_t *status;
    uint32_t *counters;   // 2 tile counters (count pass, write pass)
    const uint32_t *run;  // optional device run header {nq, nreq}: sizes read at run time (graphs)
};

struct PipeCaps {
    uint64_t nq = 0, units = 0, groups = 0, tiles = 0, rows = ~0ull;
    uint32_t nreq = 1;
    uint32_t tile = PK_TILE;  // records per tile (multiple of PK_CH)
    int pair_blocks = 0;      // pair kernel grid (0 = all resident blocks)
    uint64_t scratch = 0;     // hits the count pass keeps for placement (0: the write pass sweeps)
    uint64_t stall_ns = 0;    // plain searches only, tests of the timeout path (inject_stall)
};
constexpr uint64_t SCRATCH_MAX = 1ull << 24;  // rows (32 B each)

// Result of one search (device arrays owned by the ts_result handle).
struct SearchOut {
    uint64_t count = 0;
    uint32_t *q = nullptr, *e = nullptr;
    double *tin = nullptr, *tout = nullptr;
    ts_search_stats stats{};
};

const char *last_error();
unsigned long long launch_count();

// Plain search (R = 1) with exact-size allocations; synchronises the stream.
ts_status search_plain(const Index *ix, const ts_segments *q, const ts_query_params *qp,
                       cudaStream_t s, SearchOut *out);
ts_status measure_alu_peaks(double *fp32_tflops, double *fp64_tflops);
ts_status eval_estimates(const double *x, uint64_t n, double *rcp_est, double *sqrt_est,
                         double *rcp_ref, double *sqrt_ref);
ts_status search_points(const Index *ix, const double *x, const double *y, const double *z,
                        uint64_t n, bool on_host, const ts_query_params *qp, cudaStream_t s,
                        SearchOut *out);
ts_status schedule_only(const Index *ix, const ts_segments *q, const ts_query_params *qp,
                        cudaStream_t s, int32_t *sel, uint64_t *lo, uint64_t *hi);

// Pipeline stages (enqueue only; no host synchronisation).
ts_status pipe_prepare(const Index *ix, const double *const cols[8], uint64_t nq,
                       const ReqDesc *reqs, uint32_t nreq, const PipeBufs &b, const PipeCaps &c,
                       cudaStream_t s);
ts_status pipe_grid_units(const Index *ix, uint64_t nq, const PipeBufs &b, const PipeCaps &c,
                          cudaStream_t s);
ts_status pipe_group(const Index *ix, const ReqDesc *reqs, uint32_t nreq, const PipeBufs &b,
                     const PipeCaps &c, bool host_tiles,
                     cudaStream_t s);
ts_status pipe_count(const Index *ix, const ReqDesc *reqs, const PipeBufs &b, const PipeCaps &c,
                     cudaStream_t s);
ts_status pipe_scan_rows(const PipeBufs &b, const PipeCaps &c, cudaStream_t s);
// Tests of the timeout path: the count pass of the next plain search stalls one warp for ns
// nanoseconds on a barrier phase that never completes, then takes the timeout path.
void inject_stall(uint64_t ns);
ts_status pipe_write(const Index *ix, const ReqDesc *reqs, const PipeBufs &b, const PipeCaps &c,
                     cudaStream_t s);
// Layout of a unit's sort key: request | array (sel_bits) | top lo_bits bits of the range start.
struct KeyFmt {
    int lo_bits = 0, lo_shift = 0, sel_bits = 0;
};
constexpr int KEY_LO_BITS = 13;
constexpr int KEY_LO_MIN = 11;
KeyFmt key_fmt(const Index *ix, uint32_t nreq);
ts_status search_brute_noalloc(const ts_segments *db, const ts_segments *q,
                               const ts_query_params *qp, uint32_t *q_idx, uint32_t *e_idx,
                               double *t_in, double *t_out, uint64_t capacity, uint64_t *count,
                               cudaStream_t s);
ts_status read_dev_status(uint32_t st);
ts_status check_query_params(const ts_query_params *qp);
void fill_req(ReqDesc &r, const ts_query_params *qp, uint32_t q_first, uint32_t q_count);
ts_status device_cols(const ts_segments *q, cudaStream_t s, DevBuf &copy, const double *cols[8]);

}  // namespace ts
