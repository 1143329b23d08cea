// ts_search.cuh -- search plan shared by the plain, batched and served paths.
#pragma once

#include "ts_index.cuh"

namespace ts {

// Pair kernel geometry: 8 warps per block; each warp owns one work tile at a time and streams
// its candidate records through two shared-memory stages of PK_CH records.
constexpr int PK_WARPS = 8;
constexpr int PK_THREADS = PK_WARPS * 32;
constexpr int PK_CH = 64;          // records per stage (2 KB)
constexpr int PK_TILE = 2048;      // candidate records per tile (multiple of PK_CH)

// Device-side header of one search (written by the grouping kernels, read by the pair kernel).
enum { HDR_NVALID = 0, HDR_NGROUPS = 1, HDR_NTILES_LO = 2, HDR_NTILES_HI = 3, HDR_N = 4 };

struct PairParams {
    // groups and tiles
    const Group *groups;
    const uint64_t *tile_base;  // ngroups + 1 (scan of tiles per group)
    const uint32_t *hdr;
    // queries (caller order) and the sorted-order map
    const uint32_t *qval;       // sorted position -> caller index
    const QueryD *qd;
    const float4 *qf;           // 2 per query: (xmin, ymin, zmin, w0), (xmax, ymax, zmax, w1)
    const uint32_t *qlo, *qhi;  // own candidate range per caller query
    // candidate record arrays by selector
    const RecF *rec[5];
    const uint32_t *ids[5];     // NULL: record position == sorted entry
    const SegD *seg;
    const uint32_t *orig;
    double dd;                  // d * d
    float d2u;                  // FP32 upper bound of d^2 (with slack)
    // outputs
    uint32_t *tile_hits;        // count pass
    const uint64_t *tile_off;   // write pass (ntiles + 1)
    uint32_t *out_q, *out_e;
    double *out_tin, *out_tout;
    unsigned long long *stats;
    uint32_t *status;
    uint32_t *tile_counter;
};

// Workspace of one plain search.
struct SearchWork {
    DevBuf qd, qf, qlo, qhi, qsel, keys, vals, flags, gid, groups, ntiles, tile_base, hdr, stats,
        status, counters, tile_hits, tile_off;
};

// Result of one search (device arrays owned by the ts_result handle).
struct SearchOut {
    uint64_t count = 0;
    uint32_t *q = nullptr, *e = nullptr;
    double *tin = nullptr, *tout = nullptr;
    ts_search_stats stats{};
};

const char *last_error();
unsigned long long launch_count();
ts_status search_plain(const Index *ix, const ts_segments *q, const ts_query_params *qp,
                       cudaStream_t s, SearchOut *out);
ts_status schedule_only(const Index *ix, const ts_segments *q, const ts_query_params *qp,
                        cudaStream_t s, int32_t *sel, uint64_t *lo, uint64_t *hi);

}  // namespace ts
