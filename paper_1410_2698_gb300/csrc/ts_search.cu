// ts_search.cu -- the search pipeline: query preparation and schedule, candidate units, groups,
// and the pair kernel with its count -> scan -> write result path.
//
// Paper mapping (Gowanlock & Casanova):
//   query preparation + schedule : the host-side schedule S of Sec. 4.2 and Sec. 4.3 and the
//                                  cell lookup of Sec. 4.1, here one device thread per query
//                                  segment (binary searches on the bins' prefix maximum replace
//                                  the carried scan; a dense cell offset array replaces the
//                                  binary search in G)
//   pair kernel                  : the compare() loop of Alg. 1-3. A warp takes a tile of up to
//                                  PK_TILE consecutive candidate records shared by a group of up
//                                  to 32 candidate ranges; each lane holds one record and the
//                                  warp loops over the group's members, so a record is fetched
//                                  once for up to 32 query segments. Results are counted,
//                                  scanned and written at fixed offsets instead of being appended
//                                  atomically to a fixed-size buffer.
//
// The pair test has three stages:
//   1. FP32 box test: time extents and the entry MBB against the query MBB expanded by d, all
//      bounds rounded outward (8 compares);
//   2. FP32 gap test: squared MBB distance accumulated rounding down against an upper bound of
//      d^2 (run only when some lane passed stage 1); a pair is dropped only when a lower bound
//      of its separation exceeds d, so no pair the FP64 test could accept is ever dropped;
//   3. the exact FP64 test on the survivors (the closed form of the interaction with explicit
//      fused multiply-adds; a hit's square root and quotients from refined hardware estimates),
//      run 32 at a time on survivors compacted with ballot/popc so the FP64 pipe runs full warps.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "ts_device.cuh"
#include "ts_search.cuh"

namespace ts {

namespace {

constexpr int TPB = 256;
inline unsigned nblk(uint64_t n)
{
    uint64_t b = (n + TPB - 1) / TPB;
    if (b == 0) b = 1;
    if (b > 65535u * 32u) b = 65535u * 32u;
    return (unsigned)b;
}

// Relative slack added to the d-expanded query extents before they are mapped to subbins or grid
// cells, so FP64 rounding of (min - d) can never exclude a cell that holds a pair within d.
constexpr double EXT_SLACK = 1e-12;

__device__ __forceinline__ uint32_t req_of(const ReqDesc *reqs, uint32_t nreq, uint32_t i)
{
    uint32_t lo = 0, hi = nreq;  // last r with q_first <= i
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (reqs[mid].q_first <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t first_pmax_above(const double *pmax, uint32_t m, double w0)
{
    uint32_t lo = 0, hi = m;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (pmax[mid] > w0) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// The part of x (as part_of) from the partition's boundary table bd[j] = lo + j*w: a first guess
// in FP32 (iwf ~ 1/w; 0 when w = 0), corrected by the exact FP64 boundary comparisons, so the
// result equals part_of's.
__device__ __forceinline__ int part_of_t(double x, const double *bd, float iwf, int v)
{
    const double lo = bd[0];
    if (!(x >= lo)) return -1;
    if (v <= 1 || iwf == 0.0f) return v - 1;
    const float f = floorf((float)(x - lo) * iwf);
    int j = !(f < (float)v) ? v - 1 : (f < 0.0f ? 0 : (int)f);
    while (j + 1 < v && bd[j + 1] <= x) j++;
    while (j > 0 && bd[j] > x) j--;
    return j;
}

// First bin whose prefix maximum of B^end exceeds w0 (as first_pmax_above), searched in a bracket:
// pmax[j] >= B^start_{j+1} for every bin, so the answer is at most the bin holding w0 (jw); and
// since an entry lasts at most max_dur, bins more than `back` before jw are checked with one load
// (pmax[lo - 1] <= w0 keeps the answer at or after lo), otherwise the whole range is searched.
__device__ __forceinline__ uint32_t first_pmax_above_b(const double *pmax, const double *bs,
                                                       uint32_t m, float iwf, uint32_t back,
                                                       double w0)
{
    const int jw = part_of_t(w0, bs, iwf, (int)m);
    if (jw < 0) return first_pmax_above(pmax, 1, w0);  // before every bin: 0 or (m = 1) 1
    uint32_t hi = (uint32_t)jw + 1 < m ? (uint32_t)jw + 1 : m;
    uint32_t lo = (uint32_t)jw > back ? (uint32_t)jw - back : 0u;
    if (lo > 0 && pmax[lo - 1] > w0) lo = 0;
    // the answer lies in [lo, hi]; hi = m means no bin
    if (hi == m && !(pmax[m - 1] > w0)) return m;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (pmax[mid] > w0) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// last bin with start < w1, or -1 (the table lookup, then the strict comparison)
__device__ __forceinline__ int last_start_below_t(const double *bs, uint32_t m, float iwf,
                                                  double w1)
{
    int j = part_of_t(w1, bs, iwf, (int)m);
    while (j >= 0 && !(bs[j] < w1)) j--;
    return j;
}


// ---------------------------------------------------------------------------------------------
// query preparation (one thread per query segment of the batch)
// ---------------------------------------------------------------------------------------------
struct PrepParams {
    const double *f[8];
    uint64_t nq;
    int kind;
    const ReqDesc *reqs;
    uint32_t nreq;
    KeyFmt kf;
    // index
    uint64_t n;
    uint32_t m;
    double tmin, tmax;
    const double *bin_start, *bin_pmax;
    const uint32_t *bin_off;
    float bin_iwf;      // ~ 1 / bin width (first guesses only)
    uint32_t bin_back;  // bins an entry can reach back (from its duration), plus a margin
    uint32_t v[3];
    const double *sub_bound[3];  // subbin boundary tables (v + 1 each)
    float sub_iwf[3];
    const uint32_t *st_off[3];
    uint32_t g;
    const double *g_bound[3];    // grid boundary tables (g + 1 each)
    float g_iwf[3];
    double g_lo[3], g_w[3], longest[3];
    uint32_t smem_bytes;  // > 0: the lookup tables are first copied into shared memory
    PipeBufs b;
};

// Sort key of a unit: (request, array, range start). Only the top KEY_LO_BITS bits of the start
// are kept: the sort gathers units with nearby ranges into groups, and the groups order their
// members exactly before merging their ranges.
__device__ __forceinline__ uint64_t unit_key(uint32_t r, uint32_t sel, uint32_t lo, KeyFmt f)
{
    const uint32_t sb = f.sel_bits ? (sel & ((1u << f.sel_bits) - 1u)) : 0u;
    return ((uint64_t)r << (f.sel_bits + f.lo_bits)) | ((uint64_t)sb << f.lo_bits) |
           (uint64_t)(lo >> f.lo_shift);
}

__global__ void k_qprep(PrepParams P)
{
    // the bin, subbin and cell boundary tables the lookups read, copied into shared memory (one
    // round of loads instead of chains of dependent global loads) when they fit; they belong to
    // the index, so the copy runs before the wait on the preceding kernel
    extern __shared__ __align__(16) unsigned char qp_smem[];
    const double *bin_start = P.bin_start, *bin_pmax = P.bin_pmax;
    const uint32_t *bin_off = P.bin_off;
    const double *sub_bound[3] = {P.sub_bound[0], P.sub_bound[1], P.sub_bound[2]};
    const double *g_bound[3] = {P.g_bound[0], P.g_bound[1], P.g_bound[2]};
    if (P.smem_bytes) {
        double *sd = reinterpret_cast<double *>(qp_smem);
        const uint32_t t = threadIdx.x, nt = blockDim.x;
        if (P.kind == TS_INDEX_SPATIAL) {
            for (int d = 0; d < 3; d++) {
                for (uint32_t i = t; i <= P.g; i += nt) sd[i] = P.g_bound[d][i];
                g_bound[d] = sd;
                sd += P.g + 1;
            }
        } else {
            for (uint32_t i = t; i < P.m; i += nt) sd[i] = P.bin_start[i];
            bin_start = sd;
            sd += P.m;
            for (uint32_t i = t; i < P.m; i += nt) sd[i] = P.bin_pmax[i];
            bin_pmax = sd;
            sd += P.m;
            if (P.kind == TS_INDEX_SPATIOTEMPORAL) {
                for (int d = 0; d < 3; d++) {
                    for (uint32_t i = t; i <= P.v[d]; i += nt) sd[i] = P.sub_bound[d][i];
                    sub_bound[d] = sd;
                    sd += P.v[d] + 1;
                }
            }
            uint32_t *so = reinterpret_cast<uint32_t *>(sd);
            for (uint32_t i = t; i <= P.m; i += nt) so[i] = P.bin_off[i];
            bin_off = so;
        }
        __syncthreads();
    }
    pdl_enter();
    const uint64_t nq = P.b.run ? min((uint64_t)P.b.run[0], P.nq) : P.nq;
    const uint32_t nreq = P.b.run ? P.b.run[1] : P.nreq;
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.kind != TS_INDEX_SPATIAL)
        P.b.hdr[HDR_NU] = (uint32_t)nq;  // one unit slot per query
    uint32_t n_valid = 0, n_subbin = 0;  // (a warp's first active lane)
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = req_of(P.reqs, nreq, (uint32_t)i);
        const ReqDesc R = P.reqs[r];
        double v[8];
        bool fin = true;
        const uint64_t li = i - R.q_first;  // index within the request
#pragma unroll
        for (int k = 0; k < 8; k++) {
            v[k] = P.f[0] ? P.f[k][i] : R.cols[k][li];
            fin = fin && isfinite(v[k]);
        }
        if (!fin || !(v[7] > v[3])) atomicOr(P.b.status, DEV_ERR_INVALID);
        const double dt = v[7] - v[3];
        QueryD q;
        q.vx = (v[4] - v[0]) / dt;
        q.vy = (v[5] - v[1]) / dt;
        q.vz = (v[6] - v[2]) / dt;
        q.w0 = dmx(v[3], R.t_start);
        q.w1 = dmn(v[7], R.t_end);
        const double dw = q.w0 - v[3];  // 0 unless the request interval clips the start
        q.xw = fma(q.vx, dw, v[0]);
        q.yw = fma(q.vy, dw, v[1]);
        q.zw = fma(q.vz, dw, v[2]);
        q.ndd = -R.dd;
        q.pad = 0.0;
        const bool valid = fin && (v[7] > v[3]) && (q.w0 < q.w1);
        P.b.qd[i] = q;
        P.b.qreq[i] = r;
        double mn[3], mx[3];
        float fmn[3], fmx[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            mn[d] = v[d] < v[4 + d] ? v[d] : v[4 + d];
            mx[d] = v[d] < v[4 + d] ? v[4 + d] : v[d];
            fmn[d] = __double2float_rd(mn[d]);
            fmx[d] = __double2float_ru(mx[d]);
        }
        P.b.qf[2 * i + 0] = make_float4(__fsub_rd(fmn[0], R.d_up), __fsub_rd(fmn[1], R.d_up),
                                        __fsub_rd(fmn[2], R.d_up), __double2float_rd(q.w0));
        P.b.qf[2 * i + 1] = make_float4(__fadd_ru(fmx[0], R.d_up), __fadd_ru(fmx[1], R.d_up),
                                        __fadd_ru(fmx[2], R.d_up), __double2float_ru(q.w1));

        uint32_t sel = SEL_T, lo = 0, hi = 0;
        bool subbin = false, unit = false;
        if (P.kind == TS_INDEX_SPATIAL) {
            // cells of the grid (single assignment by MBB minimum corner) that can hold an entry
            // within d: minimum corners in [min - d - longest, max + d] per axis
            uint32_t ca[3], cb[3];
            bool any = valid;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                double a = ((mn[d] - R.d) - P.longest[d]) -
                           EXT_SLACK * ((fabs(mn[d]) + R.d) + P.longest[d]);
                double bb = (mx[d] + R.d) + EXT_SLACK * (fabs(mx[d]) + R.d);
                int pa = part_of_t(a, g_bound[d], P.g_iwf[d], (int)P.g);
                int pb = part_of_t(bb, g_bound[d], P.g_iwf[d], (int)P.g);
                if (pa < 0) pa = 0;
                if (pb < pa) any = false;
                ca[d] = (uint32_t)pa;
                cb[d] = (uint32_t)(pb < 0 ? 0 : pb);
            }
            P.b.qcell[2 * i] = ca[0] | (ca[1] << 10) | (ca[2] << 20);
            P.b.qcell[2 * i + 1] = cb[0] | (cb[1] << 10) | (cb[2] << 20);
            P.b.qnu[i] = any ? (cb[0] - ca[0] + 1) * (cb[1] - ca[1] + 1) : 0u;
        } else {
            if (valid) {
                if (P.kind == TS_INDEX_BRUTE) {
                    hi = (uint32_t)P.n;
                } else {
                    // temporal range (Sec. 4.2 schedule)
                    const uint32_t jl = first_pmax_above_b(bin_pmax, bin_start, P.m,
                                                           P.bin_iwf, P.bin_back, q.w0);
                    const int jh = last_start_below_t(bin_start, P.m, P.bin_iwf, q.w1);
                    const bool any = (int)jl <= jh;
                    if (any) {
                        lo = bin_off[jl];
                        hi = bin_off[jh + 1];
                    }
                    if (any && P.kind == TS_INDEX_SPATIOTEMPORAL) {
                        // the dimension whose d-expanded extent meets one subbin (or none) with
                        // the fewest ids over the bins jl..jh (Sec. 4.3 schedule)
                        long long best = -1;
#pragma unroll
                        for (int d = 0; d < 3; d++) {
                            const int vv = (int)P.v[d];
                            double a = (mn[d] - R.d) - EXT_SLACK * (fabs(mn[d]) + R.d);
                            double bb = (mx[d] + R.d) + EXT_SLACK * (fabs(mx[d]) + R.d);
                            const int pa = part_of_t(a, sub_bound[d], P.sub_iwf[d], vv);
                            const int pb = part_of_t(bb, sub_bound[d], P.sub_iwf[d], vv);
                            const int ja = pa < 0 ? 0 : pa, jb = pb;
                            uint32_t clo, chi;
                            if (jb < ja) {
                                clo = 0;
                                chi = 0;
                            } else if (ja == jb) {
                                const uint32_t *off = P.st_off[d];
                                clo = off[(uint64_t)ja * P.m + jl];
                                chi = off[(uint64_t)ja * P.m + jh + 1];
                            } else {
                                continue;
                            }
                            if (best < 0 || (long long)(chi - clo) < best) {
                                best = (long long)(chi - clo);
                                sel = (uint32_t)d;
                                lo = clo;
                                hi = chi;
                            }
                        }
                        subbin = best >= 0;
                    }
                }
            }
            unit = valid && hi > lo;
            P.b.u_q[i] = (uint32_t)i;
            P.b.u_lo[i] = lo;
            P.b.u_hi[i] = hi;
            P.b.u_sel[i] = sel;
            P.b.keys[i] = unit ? unit_key(r, sel, lo, P.kf) : ~0ull;
            P.b.vals[i] = (uint32_t)i;
        }
        const unsigned am = __activemask();
        const unsigned vm = __ballot_sync(am, valid);
        const unsigned sm = __ballot_sync(am, subbin);
        const int lane = threadIdx.x & 31;
        if (P.kind != TS_INDEX_SPATIAL) {
            // units per request: one atomic per request present in the warp (requests are
            // contiguous runs of queries, so nearly always one)
            const unsigned peers = __match_any_sync(am, r);
            const unsigned um = __ballot_sync(am, unit) & peers;
            if (um && lane == __ffs(peers) - 1) atomicAdd(&P.b.req_units[r], (uint32_t)__popc(um));
        }
        if (lane == __ffs(am) - 1) {
            n_valid += __popc(vm);
            n_subbin += __popc(sm);
        }
    }
    // the block's counts: one atomic per counter and block
    __shared__ uint32_t red[2][32];
    const int warp = threadIdx.x >> 5, lane0 = threadIdx.x & 31;
    for (int o = 16; o; o >>= 1) {
        n_valid += __shfl_xor_sync(0xffffffffu, n_valid, o);
        n_subbin += __shfl_xor_sync(0xffffffffu, n_subbin, o);
    }
    if (lane0 == 0) {
        red[0][warp] = n_valid;
        red[1][warp] = n_subbin;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        unsigned long long v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[threadIdx.x][w];
        if (v) atomicAdd(&P.b.stats[threadIdx.x == 0 ? ST_QSEGS : ST_SUBBIN], v);
    }
}

// Grid index: one unit per (cx, cy) of a query's cell box, covering cells cz_a..cz_b (a z-run
// of the row-major cell order, contiguous in the lookup array).
// One warp per 32 consecutive query segments: the lanes first load their query's cell box and
// unit slots (query i owns slots quoff[i] .. quoff[i] + qnu[i] - 1, so the warp's slots are one
// contiguous range), then run over the warp's slots 32 at a time, each lane finding the query of
// its slot among the lanes' starts; the unit counts per request are summed in the warp.
__global__ void k_grid_units(uint64_t nqcap, uint64_t ucap, KeyFmt kf, uint32_t g,
                             const uint32_t *g_off, PipeBufs b)
{
    pdl_enter();
    const unsigned FULL = 0xffffffffu;
    const uint64_t nq = b.run ? min((uint64_t)b.run[0], nqcap) : nqcap;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        b.hdr[HDR_NU] = (uint32_t)min((uint64_t)b.quoff[nq], ucap);  // unit slots of the runs
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < nq;
         w += warps) {
        const uint64_t i = w * 32 + lane;
        const bool has = i < nq;
        const uint32_t nu = has ? b.qnu[i] : 0u;
        // lanes past the last query start beyond every slot
        const uint32_t u0 = has ? b.quoff[i] : 0xffffffffu;
        const uint32_t r = has ? b.qreq[i] : 0u;
        const uint32_t c0 = has ? b.qcell[2 * i] : 0u, c1 = has ? b.qcell[2 * i + 1] : 0u;
        const int last = (int)min((uint64_t)31, nq - 1 - w * 32);
        const uint32_t ubeg = __shfl_sync(FULL, u0, 0);
        const uint32_t uend = __shfl_sync(FULL, u0 + nu, last);
        uint32_t cr = 0, cn = 0;  // this lane's running (request, valid units)
        for (uint32_t base = ubeg; base < uend; base += 32) {
            const uint32_t u = base + (uint32_t)lane;
            // the last lane whose start is at or before u owns slot u (a query without slots
            // shares its start with the next query, which then owns it)
            int j = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const uint32_t cand = __shfl_sync(FULL, u0, j + step);
                if (cand <= u) j += step;
            }
            const uint32_t ju0 = __shfl_sync(FULL, u0, j);
            const uint32_t jr = __shfl_sync(FULL, r, j);
            const uint32_t w0 = __shfl_sync(FULL, c0, j), w1 = __shfl_sync(FULL, c1, j);
            if (u >= uend) continue;
            if (u >= ucap) {  // more runs than the unit buffers hold
                atomicOr(b.status, DEV_ERR_OVERFLOW);
                continue;
            }
            const uint32_t ax = w0 & 1023u, ay = (w0 >> 10) & 1023u, az = (w0 >> 20) & 1023u;
            const uint32_t by = (w1 >> 10) & 1023u, bz = (w1 >> 20) & 1023u;
            const uint32_t ny = by - ay + 1;
            const uint32_t c = u - ju0;
            const uint32_t cx = ax + c / ny, cy = ay + c % ny;
            const uint64_t row = ((uint64_t)cx * g + cy) * g;
            const uint32_t lo = g_off[row + az], hi = g_off[row + bz + 1];
            b.u_q[u] = (uint32_t)(w * 32 + (uint64_t)j);
            b.u_lo[u] = lo;
            b.u_hi[u] = hi;
            b.u_sel[u] = SEL_GRID;
            b.keys[u] = hi > lo ? unit_key(jr, SEL_GRID, lo, kf) : ~0ull;
            b.vals[u] = u;
            if (jr != cr) {  // a request boundary inside the warp's slots (rare)
                if (cn) atomicAdd(&b.req_units[cr], cn);
                cr = jr;
                cn = 0;
            }
            cn += hi > lo;
        }
        // nearly always one request per warp: one atomic for the warp
        const uint32_t r0 = __shfl_sync(FULL, cr, 0);
        if (__all_sync(FULL, cr == r0 || cn == 0)) {
            uint32_t tot = cn;
            for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
            if (lane == 0 && tot) atomicAdd(&b.req_units[r0], tot);
        } else if (cn) {
            atomicAdd(&b.req_units[cr], cn);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// groups
// ---------------------------------------------------------------------------------------------
// Per request: unit starts (exclusive scan of its unit count) and group starts (ceil(units/32)).
__global__ void k_req_scan(uint32_t nreq_cap, PipeBufs b)
{
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t nreq = b.run ? min(b.run[1], nreq_cap) : nreq_cap;
    uint32_t us = 0, gs = 0;
    for (uint32_t r = 0; r < nreq; r++) {
        b.ustart[r] = us;
        b.gstart[r] = gs;
        const uint32_t n = b.req_units[r];
        const uint32_t ng = (n + GROUP - 1) / GROUP;
        b.req_groups[r] = ng;
        us += n;
        gs += ng;
    }
    b.ustart[nreq] = us;
    b.gstart[nreq] = gs;
    b.hdr[HDR_U] = us;
    b.hdr[HDR_G] = gs;
}

// One warp per group: lane p holds the group's member p; the members are ordered by (array,
// start) with a bitonic network over the lanes, and their ranges are merged into disjoint
// segments (a member opens a segment when its start lies beyond every earlier range of its
// array); each segment is cut into tiles of `tile` records.
__global__ void k_groups(uint32_t nreq_cap, uint64_t gcap, uint32_t tile, uint32_t align_sels,
                         const ReqDesc *reqs, PipeBufs b)
{
    pdl_enter();
    // (also writes the members' records, in the group's order, for the pair kernel)
    const unsigned FULL = 0xffffffffu;
    const uint32_t nreq = b.run ? min(b.run[1], nreq_cap) : nreq_cap;
    const uint32_t G = b.hdr[HDR_G];
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < gcap;
         g += warps) {
        if (g >= G) {
            if (lane == 0) b.ntiles[g] = 0;
            continue;
        }
        uint32_t lo = 0, hi = nreq;  // last r with gstart[r] <= g
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (b.gstart[mid] <= g) lo = mid; else hi = mid;
        }
        const uint32_t r = lo;
        const uint32_t first = b.ustart[r] + GROUP * ((uint32_t)g - b.gstart[r]);
        const uint32_t end = min(first + GROUP, b.ustart[r] + b.req_units[r]);
        const uint32_t n = end - first;
        if (lane == 0) {
            b.g_first[g] = first;
            b.g_count[g] = n;
            const ReqDesc &R = reqs[r];
            b.ghdr[g] = make_float4(R.d_dn, R.d2u, __uint_as_float(R.q_first), __uint_as_float(r));
        }
        // key = (array, start); lanes past the group's members hold the largest key
        uint64_t key = ~0ull;
        uint32_t mh = 0, mu = 0;
        if ((uint32_t)lane < n) {
            const uint32_t u = b.vals[first + lane];
            mu = u;
            const uint32_t us = b.u_sel[u];
            uint32_t ul = b.u_lo[u];
            if ((align_sels >> us) & 1u) ul &= ~(uint32_t)(PK_CH - 1);  // chunk-aligned tiles
            key = ((uint64_t)us << 32) | ul;
            mh = b.u_hi[u];
        }
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint64_t ok = __shfl_xor_sync(FULL, key, j);
                const uint32_t oh = __shfl_xor_sync(FULL, mh, j);
                const uint32_t ou = __shfl_xor_sync(FULL, mu, j);
                const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
                if (keep_min ? (ok < key) : (ok > key)) {
                    key = ok;
                    mh = oh;
                    mu = ou;
                }
            }
        }
        const bool member = (uint32_t)lane < n;
        const uint32_t sel = (uint32_t)(key >> 32), ml = (uint32_t)key;
        if (member) {
            MemberRec mr;
            mr.qi = b.u_q[mu];
            mr.lo = b.u_lo[mu];
            mr.hi = b.u_hi[mu];
            mr.sel = sel;
            mr.ea = b.qf[2 * (uint64_t)mr.qi + 0];
            mr.eb = b.qf[2 * (uint64_t)mr.qi + 1];
            b.gmem[(uint64_t)g * GROUP + lane] = mr;
        }
        // running maximum of the range ends over the earlier members of the same array
        uint32_t run = mh;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, run, o);
            const uint32_t vs = __shfl_up_sync(FULL, sel, o);
            if (lane >= o && vs == sel) run = max(run, v);
        }
        const uint32_t prev_run = __shfl_up_sync(FULL, run, 1);
        const uint32_t prev_sel = __shfl_up_sync(FULL, sel, 1);
        const bool start = member && (lane == 0 || prev_sel != sel || ml > prev_run);
        const unsigned starts = __ballot_sync(FULL, start);
        const unsigned nmask = n >= 32 ? FULL : ((1u << n) - 1u);
        const unsigned ends = n ? (((starts >> 1) | (1u << (n - 1))) & nmask) : 0u;
        // segment k ends at the lane before the next start (or at the last member)
        const bool is_end = n > 0 && ((ends >> lane) & 1u);
        const uint32_t a = 31 - __clz(starts & (lane == 31 ? FULL : ((2u << lane) - 1u)));
        const uint32_t seg_lo = __shfl_sync(FULL, ml, a & 31);
        const uint32_t ntile = is_end ? (run - seg_lo + tile - 1) / tile : 0u;
        uint32_t incl = ntile;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (is_end) {
            const uint32_t k = __popc(starts & (lane == 31 ? FULL : ((2u << lane) - 1u))) - 1;
            const uint64_t o = (uint64_t)g * GROUP + k;
            b.seg_lo[o] = seg_lo;
            b.seg_hi[o] = run;
            b.seg_sel[o] = sel;
            b.seg_t0[o] = incl - ntile;
        }
        if (lane == 31) {
            b.g_nseg[g] = __popc(starts);
            b.ntiles[g] = incl;
        }
    }
}

__global__ void k_hdr(uint64_t gcap, uint64_t tcap, PipeBufs b)
{
    pdl_enter();
    const uint64_t T = b.tile_base[min((uint64_t)b.hdr[HDR_G], gcap)];
    b.hdr[HDR_T_LO] = (uint32_t)T;
    b.hdr[HDR_T_HI] = (uint32_t)(T >> 32);
    b.stats[ST_GROUPS] = b.hdr[HDR_G];
    b.stats[ST_TILES] = T;
    if (T > tcap || T > PK_MAX_TILES) atomicOr(b.status, DEV_ERR_OVERFLOW);
}

// One descriptor per tile (a warp per group, lanes over the tiles of each merged segment), so
// that the pair kernel finds a tile's group, records and request with a single load.
__global__ void k_tile_desc(uint64_t gcap, uint64_t tcap, uint32_t tile, PipeBufs b)
{
    pdl_enter();
    const uint32_t G = b.hdr[HDR_G];
    const uint64_t T = b.tile_base[min((uint64_t)G, gcap)];
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // the run header's tile count (as k_hdr)
        b.hdr[HDR_T_LO] = (uint32_t)T;
        b.hdr[HDR_T_HI] = (uint32_t)(T >> 32);
        b.stats[ST_GROUPS] = G;
        b.stats[ST_TILES] = T;
        if (T > tcap || T > PK_MAX_TILES) atomicOr(b.status, DEV_ERR_OVERFLOW);
    }
    if (T > tcap || T > PK_MAX_TILES) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G && g < gcap;
         g += warps) {
        const uint32_t count = b.g_count[g];
        if (!count) continue;
        const uint32_t r = __float_as_uint(b.ghdr[g].w);
        const uint64_t base = b.tile_base[g];
        const uint32_t nseg = b.g_nseg[g];
        // lane k holds segment k (one round of loads for all the group's segments)
        uint32_t slo = 0, shi = 0, ssel = 0, st0 = 0;
        if ((uint32_t)lane < nseg) {
            const uint64_t o = (uint64_t)g * GROUP + lane;
            slo = b.seg_lo[o];
            shi = b.seg_hi[o];
            ssel = b.seg_sel[o];
            st0 = b.seg_t0[o];
        }
        for (uint32_t k = 0; k < nseg; k++) {
            const uint32_t lo = __shfl_sync(FULL, slo, k), hi = __shfl_sync(FULL, shi, k);
            const uint32_t sel = __shfl_sync(FULL, ssel, k), t0 = __shfl_sync(FULL, st0, k);
            const uint32_t n = (hi - lo + tile - 1) / tile;
            for (uint32_t j = lane; j < n; j += 32) {
                const uint32_t s0 = lo + j * tile;
                const uint32_t s1 = min(hi, s0 + tile);
                b.tdesc[base + t0 + j] =
                    make_uint4((uint32_t)g, s0, s1, sel | ((count - 1) << 3) | (r << 8));
                b.tile_hits[base + t0 + j] = 0;  // the count pass adds to it
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// pair kernel
// ---------------------------------------------------------------------------------------------
struct __align__(16) WarpSmem {
    RecF stage[PK_STAGES][PK_CH];
    MemberRec mem[GROUP];  // the tile's group members
    float4 ghdr;           // their request's d_dn, d2u, q_first (and the request)
    uint4 dnext;           // the next tile's descriptor (asynchronous copy during the sweep)
    RecF cbox[32];         // bounding records of the tile's chunks (arrays that have them)
    // exact-test queue, first in first out, carried from tile to tile: query index in the batch,
    // entry position in its sorted array, tile | sel << 29, query index within its request
    uint32_t q_qi[PK_QUEUE], q_pos[PK_QUEUE], q_tile[PK_QUEUE], q_ql[PK_QUEUE];
    uint32_t plist[PK_PLIST];  // (member << 8 | slot) pairs of a chunk that passed the box test
    unsigned long long bar[PK_STAGES];
    unsigned long long mbar;  // members + chunk boxes
    unsigned long long xbar;  // injected stall (tests): a barrier nothing ever arrives on
    // counts of the count pass: chunks, bitmask chunks, sparse member visits, survivors (then,
    // at the end, the warp's tests, FP64 tests and hits; the last slot pads to 64 bytes)
    unsigned long long sweep[8];
};

enum { PASS_COUNT = 0, PASS_WRITE = 1 };

// Flag in a tile descriptor's group word, set by the count pass on a tile with a hit that the
// scratch did not keep: the write pass sweeps exactly the flagged tiles (k_place writes the rows
// of the kept hits, the same rows the sweep gives them).
constexpr uint32_t TILE_REDO = 0x80000000u;

struct PairParams {
    PipeBufs b;
    const ReqDesc *reqs;
    const RecF *rec[5];
    const uint32_t *ids[5];
    const RecF *box[5];  // bounding record per aligned chunk of 64 records, or null
    const SegD *seg;
    const uint32_t *orig;
    uint64_t tcap;
    uint64_t rows_cap;  // write pass: rows beyond this capacity are not written (flagged)
    uint64_t scap;      // hits the count pass keeps for placement (0: none)
    uint32_t tile;      // records per tile
    // > 0 (tests only): the first warp of block 0 waits this long on a barrier phase that never
    // completes before taking any tile, so the kernel's timeout path runs (status, return)
    uint64_t stall_ns;
};

// Exact FP64 test of one (query, entry) pair and, when `interval`, its hit interval. Not inlined:
// the pair kernel calls it only for the candidates that passed both FP32 filters, so the registers
// it needs are saved around the call instead of being reserved across the whole sweep.
__device__ __noinline__ bool exact_test(const QueryD *qp, const SegD *ep, bool interval,
                                        double *tin, double *tout)
{
    const SegD e = *ep;
    const QueryD q = *qp;
    Quad qd;
    return pair_quad(q, e, qd) && quad_solve(qd, interval, tin, tout);
}

// Persistent pair kernel. Warps take tiles (a group of up to 32 query units and up to `tile`
// consecutive entries of one sorted array): the first by their index in the grid, the rest from
// a device counter. Entry records stream through
// a ring of PK_STAGES shared-memory buffers filled by 1-D bulk copies. The conservative FP32
// filters pick the candidates of the exact FP64 test; those wait in a per-warp queue that is
// carried across tiles and drained 32 at a time, so that the FP64 instructions run on full warps.
// Count pass: hits per tile. Write pass: the rows of every tile with hits, at its offset from the
// scan, in queue order (the same order in both passes, so the offsets match).
template <int PASS>
__global__ void __launch_bounds__(PK_THREADS, PK_MIN_BLOCKS) k_pair(PairParams P)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    WarpSmem &W = reinterpret_cast<WarpSmem *>(smem_raw)[wid];
    const unsigned FULL = 0xffffffffu;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const PipeBufs &B = P.b;

    if (lane == 0) {
        for (int k = 0; k < 4; k++) W.sweep[k] = 0;
        for (int k = 0; k < PK_STAGES; k++) mbar_init(&W.bar[k], 1);
        mbar_init(&W.mbar, 1);
        mbar_init(&W.xbar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity[PK_STAGES], mparity = 0u;
    bool pending[PK_STAGES], mpending = false;
#pragma unroll
    for (int k = 0; k < PK_STAGES; k++) {
        parity[k] = 0u;
        pending[k] = false;
    }
    bool abort = false;
    if (P.stall_ns && blockIdx.x == 0 && wid == 0)
        abort = !mbar_wait_bounded(&W.xbar, 0u, P.stall_ns);  // (never arrived on: times out)

    uint64_t ntiles = (uint64_t)B.hdr[HDR_T_LO] | ((uint64_t)B.hdr[HDR_T_HI] << 32);
    if (ntiles > P.tcap || ntiles > PK_MAX_TILES) ntiles = 0;  // overflow already flagged
    if (PASS == PASS_WRITE && P.scap && B.stats[ST_SCRATCH] <= P.scap)
        ntiles = 0;  // the count pass kept every hit: k_place writes the rows
    // (otherwise the write pass sweeps only the tiles whose hits were not all kept)
    if (PASS == PASS_WRITE && ntiles && B.tile_off[ntiles] > P.rows_cap) {
        // more rows than the output holds: write none (the caller sees the exact count)
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(B.status, DEV_ERR_OVERFLOW);
        ntiles = 0;
    }
    unsigned long long acc_tests = 0, acc_exact = 0, acc_hits = 0;
    uint32_t qn = 0;                            // queued candidates (warp-uniform)
    uint32_t wt_cur = 0xffffffffu, wt_cnt = 0;  // last tile with hits, its hits so far
    // count pass: the scratch had room after this warp's last reservation (the warp's own view:
    // reading the shared counter before every batch of exact tests would put a round trip to L2
    // in front of each)
    bool room = true;

    // Exact test of the oldest nflush queued candidates, one per lane.
    auto flush = [&](uint32_t nflush) {
        uint32_t qi = 0, pos = 0, tw = 0xffffffffu, ql = 0;
        if ((uint32_t)lane < nflush) {
            qi = W.q_qi[lane];
            pos = W.q_pos[lane];
            tw = W.q_tile[lane];
            ql = W.q_ql[lane];
        }
        __syncwarp();
        if (qn > nflush && (uint32_t)lane < qn - nflush) {
            const uint32_t j = nflush + lane;
            W.q_qi[lane] = W.q_qi[j];
            W.q_pos[lane] = W.q_pos[j];
            W.q_tile[lane] = W.q_tile[j];
            W.q_ql[lane] = W.q_ql[j];
        }
        __syncwarp();
        qn -= nflush;
        acc_exact += nflush;
        bool h = false;
        double tin = 0.0, tout = 0.0;
        uint32_t eid = 0;
        const uint32_t tile = tw & PK_MAX_TILES;
        // the count pass computes hit intervals only while the scratch still has room, as far
        // as this warp has seen (after an overflow the write pass sweeps and computes them; a
        // hit is kept only when its slot fits, so a stale view costs at most some intervals)
        const bool interval = PASS == PASS_WRITE || (P.scap != 0 && room);
        if ((uint32_t)lane < nflush) {
            const uint32_t *ids = P.ids[tw >> 29];
            eid = ids ? ids[pos] : pos;
            h = exact_test(B.qd + qi, P.seg + eid, interval, &tin, &tout);
        }
        const unsigned hm = __ballot_sync(FULL, h);
        if (!hm) return;
        acc_hits += __popc(hm);
        // hits of the same tile (the queue holds a tile's candidates contiguously, tiles in the
        // order this warp took them)
        const unsigned mine = hm & __match_any_sync(FULL, h ? tile : 0xffffffffu);
        // rank of the hit among its tile's rows (queue order, the same in both passes)
        const uint32_t rank = (tile == wt_cur ? wt_cnt : 0u) + __popc(mine & lt_mask);
        if (PASS == PASS_COUNT) {
            if (h && (mine & lt_mask) == 0) atomicAdd(&B.tile_hits[tile], (uint32_t)__popc(mine));
            if (P.scap) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&B.stats[ST_SCRATCH], (unsigned long long)__popc(hm));
                base = __shfl_sync(FULL, base, 0);
                room = base + (unsigned long long)__popc(hm) < P.scap;
                const unsigned long long slot = base + __popc(hm & lt_mask);
                const bool kept = h && slot < P.scap && interval;
                if (kept) {
                    B.s_tile[slot] = tile;
                    B.s_rank[slot] = rank;
                    B.s_q[slot] = ql;
                    B.s_e[slot] = P.orig[eid];
                    B.s_tin[slot] = tin;
                    B.s_tout[slot] = tout;
                }
                // a tile with a hit the scratch could not keep is swept again by the write pass
                const unsigned lost = __ballot_sync(FULL, h && !kept);
                if (h && !kept && (mine & lost & lt_mask) == 0)
                    atomicOr(&B.tdesc[tile].x, TILE_REDO);
            }
        } else if (h) {
            const uint64_t o = B.tile_off[tile] + rank;
            if (o < B.tile_off[tile + 1]) {
                B.out_q[o] = ql;
                B.out_e[o] = P.orig[eid];
                B.out_tin[o] = tin;
                B.out_tout[o] = tout;
            } else {
                atomicOr(B.status, DEV_ERR_INTERNAL);  // the passes disagree
            }
        }
        const int last = 31 - __clz(hm);
        const uint32_t last_tile = __shfl_sync(FULL, tile, last);
        const uint32_t last_n = __popc(__shfl_sync(FULL, mine, last));
        wt_cnt = (last_tile == wt_cur ? wt_cnt : 0u) + last_n;
        wt_cur = last_tile;
    };

    // tiles are taken from a device counter; the next index and its descriptor are fetched
    // while a tile is swept
    // (each warp's first tile is its index in the grid, so the counter only hands out the rest:
    // no burst of same-address atomics when every warp starts at once)
    const uint32_t nwarps = gridDim.x * PK_WARPS;
    uint64_t t = (uint64_t)blockIdx.x * PK_WARPS + wid;
    uint4 D = t < ntiles ? B.tdesc[t] : make_uint4(0u, 0u, 0u, 0u);
    while (!abort && t < ntiles) {
        uint64_t t_next = 0;
        if (lane == 0) t_next = nwarps + (uint64_t)atomicAdd(&B.counters[PASS], 1u);
        if (PASS == PASS_WRITE &&
            (B.tile_hits[t] == 0 || (P.scap && !(D.x & TILE_REDO)))) {
            // no rows in this tile, or every one of them was kept by the count pass
            t = __shfl_sync(FULL, t_next, 0);
            D = t < ntiles ? B.tdesc[t] : make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        const uint32_t g = D.x & ~TILE_REDO, s0 = D.y, s1 = D.z;
        const uint32_t sel = D.w & 7u, count = ((D.w >> 3) & 31u) + 1u;
        const uint32_t tw = (uint32_t)t | (sel << 29);
        const RecF *recs = P.rec[sel];
        const RecF *bx = P.box[sel];
        const uint32_t nrec = s1 - s0;
        const uint32_t nch = (nrec + PK_CH - 1) / PK_CH;
        // one bulk copy of the members (and of the chunks' bounding records), then the first two
        // chunks of records
        if (lane == 0) {
            const uint32_t mb = count * (uint32_t)sizeof(MemberRec);
            const uint32_t cb = bx ? nch * (uint32_t)sizeof(RecF) : 0u;
            mbar_arrive_tx(&W.mbar, mb + cb + (uint32_t)sizeof(float4));
            bulk_g2s(&W.ghdr, B.ghdr + g, (uint32_t)sizeof(float4), &W.mbar);
            bulk_g2s(&W.mem[0], B.gmem + (uint64_t)g * GROUP, mb, &W.mbar);
            if (bx) bulk_g2s(&W.cbox[0], bx + s0 / PK_CH, cb, &W.mbar);
            for (uint32_t c = 0; c < (uint32_t)PK_STAGES && c < nch; c++) {
                const uint32_t cs = s0 + c * PK_CH, cn = min((uint32_t)PK_CH, s1 - cs);
                mbar_arrive_tx(&W.bar[c], cn * (uint32_t)sizeof(RecF));
                bulk_g2s(&W.stage[c][0], recs + cs, cn * (uint32_t)sizeof(RecF), &W.bar[c]);
            }
        }
        mpending = true;
#pragma unroll
        for (int k = 0; k < PK_STAGES; k++) pending[k] = nch > (uint32_t)k;
        if (!mbar_wait_bounded(&W.mbar, mparity)) {
            abort = true;
            break;
        }
        mparity ^= 1u;
        mpending = false;
        // a group's members belong to one request: its d bounds for the gap filter
        const float4 GH = W.ghdr;
        const float d_dn = GH.x, d2u = GH.y;
        const uint32_t q_first = __float_as_uint(GH.z);
        // the next tile's descriptor is copied into shared memory during the sweep
        if (lane == 0 && t_next < ntiles) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(&W.dnext)),
                         "l"(B.tdesc + t_next)
                         : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        }

        // members of the group: one per lane, their expanded boxes and ranges in registers
        uint32_t lo = 0, hi = 0, myq = 0;
        float4 ea = make_float4(0.f, 0.f, 0.f, 0.f), eb = ea;
        if ((uint32_t)lane < count) {
            const MemberRec &M = W.mem[lane];
            myq = M.qi;
            lo = M.lo;
            hi = M.hi;
            if (M.sel != sel) lo = hi = 0;
            ea = M.ea;
            eb = M.eb;
            if (PASS == PASS_COUNT) {
                const uint32_t a = max(lo, s0), bnd = min(hi, s1);
                acc_tests += bnd > a ? bnd - a : 0u;
            }
        }
        // the two axes of the stage-1 sweep, those on which the array's entries are least likely
        // to meet the query: time and x for grid cells (a cell holds entries of every time), the
        // two other axes for a subbin array (its entries overlap the query in the subbin's axis
        // by construction), y and z for the x-ordered temporal bins (a chunk's entries are close
        // in x, and the chunk's bounding record has been tested already)
        const int dim = sel == SEL_GRID ? 3 : (sel == SEL_X || sel == SEL_T ? 1 : 0);
        const int dim2 = sel == SEL_GRID ? 0 : (sel == SEL_Z ? 1 : 2);
        auto comp = [](const float4 &v, int k) {
            return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
        };
        const float fa = comp(ea, dim), fb = comp(eb, dim);
        const float ga = comp(ea, dim2), gb = comp(eb, dim2);

        // a candidate that passed the filters joins the exact-test queue
        auto enqueue = [&](bool p, uint32_t qi, uint32_t pos) {
            const unsigned bm = __ballot_sync(FULL, p);
            if (bm) {
                if (p) {
                    const uint32_t j = qn + __popc(bm & lt_mask);
                    W.q_qi[j] = qi;
                    W.q_pos[j] = pos;
                    W.q_tile[j] = tw;
                    W.q_ql[j] = qi - q_first;
                }
                qn += __popc(bm);
                if (qn >= 32) {
                    __syncwarp();
                    flush(32);
                }
            }
        };

        // the chunks this lane's member meets: its range overlaps the chunk and, for an array
        // with chunk boxes, its expanded box meets the chunk's bounding record
        uint32_t mc = 0u;
        if (bx) {
            for (uint32_t c = 0; c < nch; c++) {
                const uint32_t cs = s0 + c * PK_CH, ce = min(cs + (uint32_t)PK_CH, s1);
                const bool meet = (lo < ce) & (hi > cs) & filter_box(W.cbox[c], ea, eb);
                mc |= (uint32_t)meet << c;
            }
        } else {
            for (uint32_t c = 0; c < nch; c++) {
                const uint32_t cs = s0 + c * PK_CH, ce = min(cs + (uint32_t)PK_CH, s1);
                mc |= (uint32_t)((lo < ce) & (hi > cs)) << c;
            }
        }
        // chunks to sweep, in order; the first PK_STAGES were copied already, later ones are
        // copied PK_STAGES sweeps ahead, so a chunk no member meets is neither copied nor swept
        const uint32_t need = __reduce_or_sync(FULL, mc);
        const uint32_t first =
            nch >= (uint32_t)PK_STAGES ? (1u << PK_STAGES) - 1u : (1u << nch) - 1u;
        uint32_t todo = need | first;
        uint32_t pend = todo & ~((1u << PK_STAGES) - 1u);
        for (uint32_t k = 0; todo && !abort; k++) {
            const uint32_t c = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int st = (int)(k % PK_STAGES);
            if (!mbar_wait_bounded(&W.bar[st], parity[st])) {
                abort = true;
                break;
            }
            parity[st] ^= 1u;
            pending[st] = false;
            if (PASS == PASS_COUNT && lane == 0) W.sweep[0]++;
            const uint32_t cs = s0 + c * PK_CH;
            const uint32_t cn = min((uint32_t)PK_CH, s1 - cs);
            const bool mine = (mc >> c) & 1u;
            // this lane's own range within the chunk, as bits of the 64 stage slots
            const uint32_t va = max(lo, cs), vb = min(hi, cs + cn);
            uint32_t v0 = 0u, v1 = 0u;
            if (mine && vb > va) {
                const uint32_t x = va - cs, y = vb - cs;  // 0 <= x < y <= 64
                v0 = (y >= 32 ? FULL : ((1u << y) - 1u)) & (x >= 32 ? 0u : (FULL << x));
                v1 = y <= 32 ? 0u : ((y >= 64 ? FULL : ((1u << (y - 32)) - 1u)) &
                                     (x <= 32 ? FULL : (FULL << (x - 32))));
            }
            uint32_t m0 = 0u, m1 = 0u;
            const unsigned act = __ballot_sync(FULL, (v0 | v1) != 0u);
            if (!act) {
                // (a chunk copied ahead of the member tests that no member meets)
            } else if (__popc(act) <= PK_SPARSE) {
                if (PASS == PASS_COUNT && lane == 0) W.sweep[2] += __popc(act);
                // few members meet this chunk: one lane per slot (slots lane and lane + 32), the
                // members that meet the chunk in turn, their boxes read as broadcasts
                const bool in0 = (uint32_t)lane < cn, in1 = (uint32_t)lane + 32 < cn;
                RecF r0 = W.stage[st][lane];
                RecF r1 = W.stage[st][lane + 32];
                if (!in0) r0.t0 = INFINITY;  // a slot past the chunk never passes the filter
                if (!in1) r1.t0 = INFINITY;
                const uint32_t pos0 = cs + lane, pos1 = cs + 32 + lane;
                // the (member, slot) pairs that pass the box test are listed in shared memory
                // (member by member, slot order) and go through the gap bound one per lane, so
                // that the gap bound and the queue run on full warps
                uint32_t npl = 0;  // listed pairs (warp-uniform)
                auto drain = [&]() {
                    __syncwarp();
                    for (uint32_t b = 0; b < npl; b += 32) {
                        bool p = false;
                        uint32_t mq = 0, slot = 0;
                        if (b + lane < npl) {
                            const uint32_t e = W.plist[b + lane];
                            const MemberRec &M = W.mem[e >> 8];
                            slot = e & 63u;
                            mq = M.qi;
                            p = filter_gap_e(W.stage[st][slot], M.ea, M.eb, d_dn, d2u);
                        }
                        enqueue(p, mq, cs + slot);
                    }
                    npl = 0;
                    __syncwarp();
                };
                for (unsigned rem = act; rem; rem &= rem - 1u) {
                    // (a member in act has this tile's array: its range is its own)
                    const uint32_t m = __ffs(rem) - 1;
                    const MemberRec &M = W.mem[m];
                    const float4 mea = M.ea, meb = M.eb;
                    const uint32_t mlo = M.lo;
                    const uint32_t w = M.hi - mlo;
                    const bool p0 = ((pos0 - mlo) < w) & filter_box(r0, mea, meb);
                    const bool p1 = ((pos1 - mlo) < w) & filter_box(r1, mea, meb);
                    const unsigned b0 = __ballot_sync(FULL, p0), b1 = __ballot_sync(FULL, p1);
                    if (!(b0 | b1)) continue;  // (the common case)
                    if (p0) W.plist[npl + __popc(b0 & lt_mask)] = (m << 8) | (uint32_t)lane;
                    if (p1)
                        W.plist[npl + __popc(b0) + __popc(b1 & lt_mask)] =
                            (m << 8) | (uint32_t)(lane + 32);
                    npl += __popc(b0) + __popc(b1);
                    if (npl > PK_PLIST - 64) drain();  // (room for one more member's 64 pairs)
                }
                if (npl) drain();
            } else {
                // stage 1: two axes of every slot against every member (slot i is read at a
                // warp-uniform address, a shared-memory broadcast); bit i is set when the extents
                // overlap on both. Four independent accumulators per half keep the OR chains
                // short.
                if (PASS == PASS_COUNT && lane == 0) W.sweep[1]++;
                const float2 *ax = reinterpret_cast<const float2 *>(&W.stage[st][0]) + dim;
                const float2 *ax2 = reinterpret_cast<const float2 *>(&W.stage[st][0]) + dim2;
                uint32_t a[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
                for (int i = 0; i < 64; i++) {
                    const float2 v = ax[4 * i], u = ax2[4 * i];
                    if ((v.y >= fa) & (v.x <= fb) & (u.y >= ga) & (u.x <= gb))
                        a[(i >> 5) * 4 + (i & 3)] |= 1u << (i & 31);
                }
                m0 = ((a[0] | a[1]) | (a[2] | a[3])) & v0;
                m1 = ((a[4] | a[5]) | (a[6] | a[7])) & v1;
            }
            // stage 2: the survivors, one per lane per round, through the full box and gap
            // filters and into the exact-test queue
            for (;;) {
                const bool have = (m0 | m1) != 0u;
                const unsigned hv = __ballot_sync(FULL, have);
                if (!hv) break;
                if (PASS == PASS_COUNT && lane == 0) W.sweep[3] += __popc(hv);
                bool p = false;
                uint32_t i = 0;
                if (have) {
                    if (m0) {
                        i = __ffs(m0) - 1;
                        m0 &= m0 - 1u;
                    } else {
                        i = 31 + __ffs(m1);
                        m1 &= m1 - 1u;
                    }
                    const RecF r = W.stage[st][i];
                    p = filter_box(r, ea, eb) & filter_gap_e(r, ea, eb, d_dn, d2u);
                }
                enqueue(p, myq, cs + i);
            }
            __syncwarp();
            if (pend) {
                const uint32_t cnext = __ffs(pend) - 1;
                pend &= pend - 1u;
                if (lane == 0) {
                    const uint32_t ns = s0 + cnext * PK_CH, nn = min((uint32_t)PK_CH, s1 - ns);
                    mbar_arrive_tx(&W.bar[st], nn * (uint32_t)sizeof(RecF));
                    bulk_g2s(&W.stage[st][0], recs + ns, nn * (uint32_t)sizeof(RecF), &W.bar[st]);
                }
                pending[st] = true;
            }
        }
        if (lane == 0) asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        t = __shfl_sync(FULL, t_next, 0);
        D = W.dnext;
        __syncwarp();  // (read by every lane before the next copy)
    }
    if (!abort && qn) {
        __syncwarp();
        flush(qn);
    }
    if (abort) {
        if (lane == 0) atomicOr(B.status, DEV_ERR_TIMEOUT);
        // let copies still in flight land before the shared memory is released
        for (int st = 0; st < PK_STAGES; st++)
            if (pending[st]) mbar_wait_bounded(&W.bar[st], parity[st]);
        if (mpending) mbar_wait_bounded(&W.mbar, mparity);
    }
    if (PASS == PASS_COUNT) {
        // the block's counts are summed in shared memory: one atomic per counter and block
        // (warps finish together, so per-warp atomics on these few addresses would queue)
        for (int o = 16; o; o >>= 1) acc_tests += __shfl_xor_sync(FULL, acc_tests, o);
        if (lane == 0) {
            W.sweep[4] = acc_tests;
            W.sweep[5] = acc_exact;
            W.sweep[6] = acc_hits;
        }
        __syncthreads();
        if (threadIdx.x < 7) {
            const WarpSmem *all = reinterpret_cast<const WarpSmem *>(smem_raw);
            unsigned long long v = 0;
            for (int w = 0; w < PK_WARPS; w++) v += all[w].sweep[threadIdx.x];
            const int slot = threadIdx.x < 4 ? ST_CHUNKS + (int)threadIdx.x
                                             : (threadIdx.x == 4 ? ST_TESTS
                                                                 : (threadIdx.x == 5 ? ST_EXACT
                                                                                     : ST_HITS));
            if (v) atomicAdd(&B.stats[slot], v);
        }
    }
}

// Rows of the hits the count pass kept: row = the tile's scanned offset + the hit's rank in the
// tile, the same row the write pass's sweep would give it. When the scratch overflowed, the
// tiles it could not hold are swept again by the write pass (which writes the same values to the
// rows placed here). Does nothing when the rows exceed the output capacity.
__global__ void k_place(PipeBufs b, uint64_t scap, uint64_t tcap, uint64_t rows_cap)
{
    pdl_enter();
    const unsigned long long n = min((unsigned long long)scap, b.stats[ST_SCRATCH]);
    const uint64_t T = (uint64_t)b.hdr[HDR_T_LO] | ((uint64_t)b.hdr[HDR_T_HI] << 32);
    if (T > tcap || T > PK_MAX_TILES) return;  // overflow already flagged
    if (b.tile_off[T] > rows_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(b.status, DEV_ERR_OVERFLOW);
        return;
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = b.s_tile[i];
        const uint64_t o = b.tile_off[t] + b.s_rank[i];
        if (t >= T || o >= b.tile_off[t + 1]) {
            atomicOr(b.status, DEV_ERR_INTERNAL);
            continue;
        }
        b.out_q[o] = b.s_q[i];
        b.out_e[o] = b.s_e[i];
        b.out_tin[o] = b.s_tin[i];
        b.out_tout[o] = b.s_tout[i];
    }
}

int g_pair_blocks = 0;

ts_status pair_grid(int *blocks)
{
    if (g_pair_blocks > 0) {
        *blocks = g_pair_blocks;
        return TS_OK;
    }
    int dev = 0, sms = 0, per = 0;
    TS_CUDA(cudaGetDevice(&dev));
    TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int smem = (int)sizeof(WarpSmem) * PK_WARPS;
    TS_CUDA(cudaFuncSetAttribute(k_pair<PASS_COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    TS_CUDA(cudaFuncSetAttribute(k_pair<PASS_WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    TS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<PASS_COUNT>, PK_THREADS, smem));
    if (per < 1) per = 1;
    g_pair_blocks = sms * per;
    *blocks = g_pair_blocks;
    return TS_OK;
}

void fill_pair_params(PairParams &P, const Index *ix, const ReqDesc *reqs, const PipeBufs &b,
                      const PipeCaps &c)
{
    P.b = b;
    P.reqs = reqs;
    for (int k = 0; k < 3; k++) {
        P.rec[k] = ix->st_rec[k];
        P.ids[k] = ix->st_ids[k];
    }
    // ranges over the start-time order cover whole bins: they are swept in the copy ordered by
    // x inside every bin, chunk by chunk with the chunks' bounding records
    P.rec[SEL_T] = ix->trec ? ix->trec : ix->rec;
    P.ids[SEL_T] = ix->trec ? ix->tid : nullptr;
    for (int k = 0; k < 5; k++) P.box[k] = nullptr;
    P.box[SEL_T] = ix->tbox;
    P.rec[SEL_GRID] = ix->ga_rec;
    P.ids[SEL_GRID] = ix->ga;
    P.box[SEL_GRID] = ix->gbox;
    P.seg = ix->seg;
    P.orig = ix->orig;
    P.tcap = c.tiles;
    P.rows_cap = c.rows;
    P.scap = c.scratch;
    P.tile = c.tile;
    P.stall_ns = 0;
}

// A stall requested for the next count pass (tests of the timeout path), taken by that launch.
std::atomic<uint64_t> g_stall_ns{0};

// Two CUDA events bracketing one kernel launch on its stream.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ts_status create()
    {
        TS_CUDA(cudaEventCreate(&a));
        TS_CUDA(cudaEventCreate(&b));
        return TS_OK;
    }
    double ms() const
    {
        float v = 0.f;
        if (a && b && cudaEventElapsedTime(&v, a, b) == cudaSuccess) return (double)v;
        return 0.0;
    }
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Smallest float >= x (host).
float float_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

// Largest float <= x (host).
float float_dn(double x)
{
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

int bits_for(uint64_t v)
{
    int b = 0;
    while (b < 64 && (v >> b) != 0) b++;
    return b;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// pipeline stages
// ---------------------------------------------------------------------------------------------
KeyFmt key_fmt(const Index *ix, uint32_t nreq)
{
    uint64_t maxlen = ix->n;
    for (int d = 0; d < 3; d++) maxlen = std::max<uint64_t>(maxlen, ix->st_len[d]);
    maxlen = std::max<uint64_t>(maxlen, ix->g_len);
    KeyFmt f;
    f.sel_bits = ix->kind == TS_INDEX_SPATIOTEMPORAL ? 2 : 0;  // X, Y, Z or T
    const int full = bits_for(maxlen);  // bits of a range start
    // as many start bits as keep the whole key (with the request and guard bits) within two
    // 8-bit radix passes, but no fewer than KEY_LO_MIN and no more than KEY_LO_BITS
    const int fit = 16 - 1 - f.sel_bits - bits_for(nreq > 1 ? nreq - 1 : 0);
    f.lo_bits = std::min(full, std::max(KEY_LO_MIN, std::min(KEY_LO_BITS, fit)));
    f.lo_shift = full - f.lo_bits;
    return f;
}

void fill_req(ReqDesc &r, const ts_query_params *qp, uint32_t q_first, uint32_t q_count)
{
    r.d = qp->d;
    r.dd = qp->d * qp->d;
    r.t_start = qp->t_start;
    r.t_end = qp->t_end;
    r.q_first = q_first;
    r.q_count = q_count;
    r.d_up = float_up(qp->d);
    r.d_dn = float_dn(qp->d);
    r.pad = 0.0f;
    for (int k = 0; k < 8; k++) r.cols[k] = nullptr;
    r.d2u = float_up(r.dd * (1.0 + 1e-6));
}

ts_status pipe_prepare(const Index *ix, const double *const cols[8], uint64_t nq,
                       const ReqDesc *reqs, uint32_t nreq, const PipeBufs &b, const PipeCaps &c,
                       cudaStream_t s)
{
    // cols == nullptr: every request's columns are read through its descriptor, and the run's
    // counters were reset by the caller
    if (cols) {
        TS_CUDA(cudaMemsetAsync(b.stats, 0, sizeof(unsigned long long) * ST_NSLOTS, s));
        TS_CUDA(cudaMemsetAsync(b.status, 0, sizeof(uint32_t), s));
        TS_CUDA(cudaMemsetAsync(b.counters, 0, sizeof(uint32_t) * 2, s));
        TS_CUDA(cudaMemsetAsync(b.req_units, 0, sizeof(uint32_t) * nreq, s));
    }
    PrepParams P;
    for (int k = 0; k < 8; k++) P.f[k] = cols ? cols[k] : nullptr;
    P.nq = nq;
    P.kind = ix->kind;
    P.reqs = reqs;
    P.nreq = nreq;
    P.kf = key_fmt(ix, c.nreq);
    P.n = ix->n;
    P.m = ix->m;
    P.tmin = ix->tmin;
    P.tmax = ix->tmax;
    P.bin_start = ix->bin_start;
    P.bin_pmax = ix->bin_pmax;
    P.bin_off = ix->bin_off;
    P.bin_iwf = ix->b > 0.0 ? (float)(1.0 / ix->b) : 0.0f;
    {
        const double back = ix->b > 0.0 ? ceil(ix->max_dur / ix->b) + 2.0 : (double)ix->m;
        P.bin_back = back < (double)ix->m ? (uint32_t)back : ix->m;
    }
    for (int d = 0; d < 3; d++) {
        P.v[d] = ix->v[d];
        P.sub_bound[d] = ix->sub_bound[d];
        P.sub_iwf[d] = ix->sub_w[d] > 0.0 ? (float)(1.0 / ix->sub_w[d]) : 0.0f;
        P.st_off[d] = ix->st_off[d];
        P.g_bound[d] = ix->g_bound[d];
        P.g_iwf[d] = ix->g_w[d] > 0.0 ? (float)(1.0 / ix->g_w[d]) : 0.0f;
        P.g_lo[d] = ix->g_lo[d];
        P.g_w[d] = ix->g_w[d];
        P.longest[d] = ix->longest[d];
    }
    P.g = ix->g;
    P.b = b;
    // lookup tables in shared memory when they fit the default 48 KB
    uint64_t tb = 0;
    if (ix->kind == TS_INDEX_SPATIAL) {
        tb = 3ull * 8 * ((uint64_t)ix->g + 1);
    } else if (ix->kind != TS_INDEX_BRUTE) {
        tb = 16ull * ix->m + 4ull * ((uint64_t)ix->m + 1);
        if (ix->kind == TS_INDEX_SPATIOTEMPORAL)
            for (int d = 0; d < 3; d++) tb += 8ull * ((uint64_t)ix->v[d] + 1);
    }
    P.smem_bytes = tb <= 48 * 1024 ? (uint32_t)tb : 0u;
    if (nq) {
        TS_LAUNCH_PDL(k_qprep, dim3(nblk(nq)), dim3(TPB), P.smem_bytes, s,
                      P);
    }
    return TS_OK;
}

ts_status pipe_grid_units(const Index *ix, uint64_t nq, const PipeBufs &b, const PipeCaps &c,
                          cudaStream_t s)
{
    if (!nq) return TS_OK;
    const unsigned ublk = (unsigned)std::min<uint64_t>((nq + TPB - 1) / TPB, 152 * 16);
    TS_LAUNCH_PDL(k_grid_units, dim3(ublk), dim3(TPB), 0, s,
                  nq, c.units, key_fmt(ix, c.nreq), ix->g, ix->g_off, b);
    return TS_OK;
}

ts_status pipe_group(const Index *ix, const ReqDesc *reqs, uint32_t nreq, const PipeBufs &b,
                     const PipeCaps &c, bool host_tiles,
                     cudaStream_t s)
{
    // one bit above the key fields: a unit without candidates has key ~0 and sorts last
    const KeyFmt f = key_fmt(ix, c.nreq);
    const int bits = f.lo_bits + f.sel_bits + bits_for(c.nreq > 1 ? c.nreq - 1 : 0) + 1;
    TS_CHECK(radix_sort_u64(b.keys, b.vals, c.units, bits, s, b.hdr + HDR_NU));
    TS_LAUNCH_PDL(k_req_scan, dim3(1), dim3(32), 0, s,
                  nreq, b);
    const unsigned gblk = (unsigned)std::min<uint64_t>((c.groups * 32 + TPB - 1) / TPB, 152 * 16);
    TS_LAUNCH_PDL(k_groups, dim3(gblk), dim3(TPB), 0, s,
                  nreq, c.groups, c.tile,
                  (ix->tbox ? (1u << SEL_T) : 0u) | (ix->gbox ? (1u << SEL_GRID) : 0u), reqs, b);
    TS_CHECK(scan_u32_to_u64(b.ntiles, b.tile_base, c.groups, s, b.hdr + HDR_G));
    if (host_tiles) {  // the caller reads the tile count before the count pass
        TS_LAUNCH_PDL(k_hdr, dim3(1), dim3(1), 0, s,
                      c.groups, c.tiles, b);
    }
    return TS_OK;
}

ts_status pipe_count(const Index *ix, const ReqDesc *reqs, const PipeBufs &b, const PipeCaps &c,
                     cudaStream_t s)
{
    int blocks = 0;
    TS_CHECK(pair_grid(&blocks));
    if (c.pair_blocks > 0 && c.pair_blocks < blocks) blocks = c.pair_blocks;
    PairParams P;
    fill_pair_params(P, ix, reqs, b, c);
    P.stall_ns = c.stall_ns;
    if (c.tiles) {
        const unsigned dblk = (unsigned)std::min<uint64_t>((c.groups * 32 + TPB - 1) / TPB, 152 * 16);
        TS_LAUNCH_PDL(k_tile_desc, dim3(dblk), dim3(TPB), 0, s,
                      c.groups, c.tiles, c.tile, b);
        TS_LAUNCH_PDL(k_pair<PASS_COUNT>, dim3(blocks), dim3(PK_THREADS),
                      sizeof(WarpSmem) * PK_WARPS, s, P);
    }
    return TS_OK;
}

void inject_stall(uint64_t ns) { g_stall_ns.store(ns); }

ts_status pipe_scan_rows(const PipeBufs &b, const PipeCaps &c, cudaStream_t s)
{
    return scan_u32_to_u64(b.tile_hits, b.tile_off, c.tiles, s, b.hdr + HDR_T_LO);
}

ts_status pipe_write(const Index *ix, const ReqDesc *reqs, const PipeBufs &b, const PipeCaps &c,
                     cudaStream_t s)
{
    int blocks = 0;
    TS_CHECK(pair_grid(&blocks));
    if (c.pair_blocks > 0 && c.pair_blocks < blocks) blocks = c.pair_blocks;
    PairParams P;
    fill_pair_params(P, ix, reqs, b, c);
    if (c.tiles) {
        if (c.scratch) {
            TS_LAUNCH_PDL(k_place, dim3(152 * 4), dim3(TPB), 0, s,
                          b, c.scratch, c.tiles, c.rows);
        }
        TS_LAUNCH_PDL(k_pair<PASS_WRITE>, dim3(blocks), dim3(PK_THREADS),
                      sizeof(WarpSmem) * PK_WARPS, s, P);
    }
    return TS_OK;
}

// ---------------------------------------------------------------------------------------------
// host orchestration of one plain search
// ---------------------------------------------------------------------------------------------
ts_status read_dev_status(uint32_t st)
{
    if (st & DEV_ERR_INVALID) {
        set_error("invalid query segment (NaN/Inf or t_end <= t_start)");
        return TS_ERR_INVALID_ARG;
    }
    if (st & DEV_ERR_TIMEOUT) {
        set_error("a bounded device wait ran out (bulk copy did not complete)");
        return TS_ERR_TIMEOUT;
    }
    if (st & DEV_ERR_OVERFLOW) {
        set_error("a work buffer capacity was exceeded");
        return TS_ERR_CAPACITY;
    }
    if (st) {
        set_error("search: device status 0x%x", st);
        return TS_ERR_INTERNAL;
    }
    return TS_OK;
}

ts_status device_cols(const ts_segments *q, cudaStream_t s, DevBuf &copy, const double *cols[8])
{
    const double *src[8] = {q->x0, q->y0, q->z0, q->t0, q->x1, q->y1, q->z1, q->t1};
    for (int k = 0; k < 8; k++)
        if (!src[k] && q->n) {
            set_error("NULL query column %d", k);
            return TS_ERR_INVALID_ARG;
        }
    if (!q->on_host) {
        for (int k = 0; k < 8; k++) cols[k] = src[k];
        return TS_OK;
    }
    TS_CHECK(copy.alloc(sizeof(double) * q->n * 8, s));
    for (int k = 0; k < 8; k++) {
        double *dst = copy.as<double>() + (uint64_t)k * q->n;
        TS_CUDA(cudaMemcpyAsync(dst, src[k], sizeof(double) * q->n, cudaMemcpyHostToDevice, s));
        cols[k] = dst;
    }
    return TS_OK;
}

ts_status check_query_params(const ts_query_params *qp)
{
    if (!qp) {
        set_error("NULL query parameters");
        return TS_ERR_INVALID_ARG;
    }
    if (!(qp->d > 0.0) || !isfinite(qp->d)) {
        set_error("d must be finite and > 0 (got %g)", qp->d);
        return TS_ERR_INVALID_ARG;
    }
    if (isnan(qp->t_start) || isnan(qp->t_end) || qp->t_start > qp->t_end) {
        set_error("query interval must satisfy t_start <= t_end");
        return TS_ERR_INVALID_ARG;
    }
    return TS_OK;
}

namespace {

// Work buffers of a plain search, allocated stage by stage at their exact sizes.
struct PlainWork {
    DevBuf qd, qf, qreq, qcell, qnu, quoff, u_q, u_lo, u_hi, u_sel, keys, vals, req, groups, segs,
        ntiles, tile_base, tiles, tdesc, tile_off, ctl, reqdesc, scratch, gmem;
};

ts_status alloc_units(PlainWork &w, PipeBufs &b, uint64_t units, cudaStream_t s)
{
    TS_CHECK(w.u_q.alloc(sizeof(uint32_t) * units, s));
    TS_CHECK(w.u_lo.alloc(sizeof(uint32_t) * units, s));
    TS_CHECK(w.u_hi.alloc(sizeof(uint32_t) * units, s));
    TS_CHECK(w.u_sel.alloc(sizeof(uint32_t) * units, s));
    TS_CHECK(w.keys.alloc(sizeof(uint64_t) * units, s));
    TS_CHECK(w.vals.alloc(sizeof(uint32_t) * units, s));
    b.u_q = w.u_q.as<uint32_t>();
    b.u_lo = w.u_lo.as<uint32_t>();
    b.u_hi = w.u_hi.as<uint32_t>();
    b.u_sel = w.u_sel.as<uint32_t>();
    b.keys = w.keys.as<uint64_t>();
    b.vals = w.vals.as<uint32_t>();
    return TS_OK;
}

ts_status plain_prepare(const Index *ix, const double *const cols[8], uint64_t nq,
                        const ts_query_params *qp, cudaStream_t s, PlainWork &w, PipeBufs &b,
                        PipeCaps &c, bool group)
{
    b = PipeBufs{};
    c = PipeCaps{};
    c.nq = nq;
    c.nreq = 1;
    ReqDesc rd;
    fill_req(rd, qp, 0, (uint32_t)nq);
    TS_CHECK(w.reqdesc.alloc(sizeof(ReqDesc), s));
    TS_CUDA(cudaMemcpyAsync(w.reqdesc.p, &rd, sizeof(ReqDesc), cudaMemcpyHostToDevice, s));
    TS_CHECK(w.qd.alloc(sizeof(QueryD) * nq, s));
    TS_CHECK(w.qf.alloc(sizeof(float4) * 2 * nq, s));
    TS_CHECK(w.qreq.alloc(sizeof(uint32_t) * nq, s));
    // control block: hdr (8 u32), stats (ST_NSLOTS u64), status, 2 counters
    TS_CHECK(w.ctl.alloc(256, s));
    TS_CHECK(w.req.alloc(sizeof(uint32_t) * 8, s));
    b.qd = w.qd.as<QueryD>();
    b.qf = w.qf.as<float4>();
    b.qreq = w.qreq.as<uint32_t>();
    b.hdr = w.ctl.as<uint32_t>();
    b.stats = reinterpret_cast<unsigned long long *>(w.ctl.as<uint32_t>() + 8);
    b.status = w.ctl.as<uint32_t>() + 8 + 2 * ST_NSLOTS;
    b.counters = b.status + 1;
    b.req_units = w.req.as<uint32_t>();
    b.ustart = b.req_units + 1;
    b.req_groups = b.req_units + 3;
    b.gstart = b.req_units + 4;
    uint64_t units = nq;
    if (ix->kind == TS_INDEX_SPATIAL) {
        TS_CHECK(w.qcell.alloc(sizeof(uint32_t) * 2 * nq, s));
        TS_CHECK(w.qnu.alloc(sizeof(uint32_t) * nq, s));
        TS_CHECK(w.quoff.alloc(sizeof(uint32_t) * (nq + 1), s));
        b.qcell = w.qcell.as<uint32_t>();
        b.qnu = w.qnu.as<uint32_t>();
        b.quoff = w.quoff.as<uint32_t>();
    } else {
        TS_CHECK(alloc_units(w, b, nq, s));
    }
    TS_CHECK(pipe_prepare(ix, cols, nq, w.reqdesc.as<ReqDesc>(), 1, b, c, s));
    if (ix->kind == TS_INDEX_SPATIAL) {
        TS_CHECK(scan_u32(b.qnu, b.quoff, nq, b.status, s));
        uint32_t total = 0;
        TS_CUDA(cudaMemcpyAsync(&total, b.quoff + nq, 4, cudaMemcpyDeviceToHost, s));
        TS_CUDA(cudaStreamSynchronize(s));
        units = total;
        TS_CHECK(alloc_units(w, b, units, s));
        c.units = units;
        TS_CHECK(pipe_grid_units(ix, nq, b, c, s));
    }
    c.units = units;
    if (!group) return TS_OK;
    c.groups = (units + GROUP - 1) / GROUP + 1;
    TS_CHECK(w.groups.alloc(sizeof(uint32_t) * 3 * c.groups, s));
    TS_CHECK(w.gmem.alloc((sizeof(MemberRec) * GROUP + sizeof(float4)) * c.groups, s));
    b.gmem = w.gmem.as<MemberRec>();
    b.ghdr = reinterpret_cast<float4 *>(b.gmem + GROUP * c.groups);
    TS_CHECK(w.segs.alloc(sizeof(uint32_t) * 4 * GROUP * c.groups, s));
    TS_CHECK(w.ntiles.alloc(sizeof(uint32_t) * c.groups, s));
    TS_CHECK(w.tile_base.alloc(sizeof(uint64_t) * (c.groups + 1), s));
    b.g_first = w.groups.as<uint32_t>();
    b.g_count = b.g_first + c.groups;
    b.g_nseg = b.g_count + c.groups;
    b.seg_lo = w.segs.as<uint32_t>();
    b.seg_hi = b.seg_lo + GROUP * c.groups;
    b.seg_sel = b.seg_hi + GROUP * c.groups;
    b.seg_t0 = b.seg_sel + GROUP * c.groups;
    b.ntiles = w.ntiles.as<uint32_t>();
    b.tile_base = w.tile_base.as<uint64_t>();
    c.tiles = ~0ull;  // sized after the grouping; no overflow check in the header kernel
    TS_CHECK(pipe_group(ix, w.reqdesc.as<ReqDesc>(), 1, b, c, true, s));
    return TS_OK;
}

ts_status copy_stats(const PipeBufs &b, cudaStream_t s, ts_search_stats *st, uint32_t *status)
{
    unsigned long long h[ST_NSLOTS];
    TS_CUDA(cudaMemcpyAsync(h, b.stats, sizeof(h), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(status, b.status, 4, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    st->n_qsegs = h[ST_QSEGS];
    st->n_tests = h[ST_TESTS];
    st->n_exact = h[ST_EXACT];
    st->n_hits = h[ST_HITS];
    st->n_tiles = h[ST_TILES];
    st->n_groups = h[ST_GROUPS];
    st->n_subbin = h[ST_SUBBIN];
    st->n_chunks = h[ST_CHUNKS];
    st->n_dense = h[ST_DENSE];
    st->n_sparse = h[ST_SPARSE];
    st->n_stage2 = h[ST_STAGE2];
    return TS_OK;
}

}  // namespace

ts_status search_plain(const Index *ix, const ts_segments *q, const ts_query_params *qp,
                       cudaStream_t s, SearchOut *out)
{
    TS_CHECK(check_query_params(qp));
    if (!q) {
        set_error("NULL query set");
        return TS_ERR_INVALID_ARG;
    }
    if (q->n > 0x7fffffffull) {
        set_error("query set larger than 2^31 - 1 segments");
        return TS_ERR_INVALID_ARG;
    }
    *out = SearchOut{};
    const uint64_t nq = q->n;
    out->stats.n_queries = nq;
    if (nq == 0) return TS_OK;
    DevBuf qcopy;
    const double *cols[8];
    TS_CHECK(device_cols(q, s, qcopy, cols));
    PlainWork w;
    PipeBufs b;
    PipeCaps c;
    TS_CHECK(plain_prepare(ix, cols, nq, qp, s, w, b, c, true));

    uint32_t hdr[HDR_N];
    uint32_t st = 0;
    TS_CUDA(cudaMemcpyAsync(hdr, b.hdr, sizeof(hdr), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(&st, b.status, 4, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    TS_CHECK(read_dev_status(st));
    c.tiles = (uint64_t)hdr[HDR_T_LO] | ((uint64_t)hdr[HDR_T_HI] << 32);
    TS_CHECK(w.tiles.alloc(sizeof(uint32_t) * (c.tiles ? c.tiles : 1), s));
    TS_CHECK(w.tdesc.alloc(sizeof(uint4) * (c.tiles ? c.tiles : 1), s));
    TS_CHECK(w.tile_off.alloc(sizeof(uint64_t) * (c.tiles + 1), s));
    b.tdesc = w.tdesc.as<uint4>();
    b.tile_hits = w.tiles.as<uint32_t>();
    // hits kept by the count pass and placed after the scan (a second sweep when they overflow)
    c.scratch = std::min<uint64_t>(4 * nq + (1ull << 20), SCRATCH_MAX);
    TS_CHECK(w.scratch.alloc(32 * c.scratch, s));
    b.s_tile = w.scratch.as<uint32_t>();
    b.s_rank = b.s_tile + c.scratch;
    b.s_q = b.s_rank + c.scratch;
    b.s_e = b.s_q + c.scratch;
    b.s_tin = reinterpret_cast<double *>(b.s_e + c.scratch);
    b.s_tout = b.s_tin + c.scratch;
    b.tile_off = w.tile_off.as<uint64_t>();

    EventPair ev_count, ev_write;
    TS_CHECK(ev_count.create());
    TS_CHECK(ev_write.create());
    c.stall_ns = g_stall_ns.exchange(0);  // (a stall requested by a test of the timeout path)
    TS_CUDA(cudaEventRecord(ev_count.a, s));
    TS_CHECK(pipe_count(ix, w.reqdesc.as<ReqDesc>(), b, c, s));
    TS_CUDA(cudaEventRecord(ev_count.b, s));
    TS_CHECK(pipe_scan_rows(b, c, s));
    uint64_t total = 0;
    TS_CUDA(cudaMemcpyAsync(&total, b.tile_off + c.tiles, 8, cudaMemcpyDeviceToHost, s));
    TS_CHECK(copy_stats(b, s, &out->stats, &st));
    TS_CHECK(read_dev_status(st));
    out->stats.n_queries = nq;
    out->stats.ms_count_pass = ev_count.ms();
    out->count = total;
    if (out->stats.n_hits != total) {
        set_error("hit count mismatch (%llu vs %llu)", (unsigned long long)out->stats.n_hits,
                  (unsigned long long)total);
        return TS_ERR_INTERNAL;
    }
    if (qp->max_results && total > qp->max_results) {
        set_error("%llu result rows exceed max_results %llu", (unsigned long long)total,
                  (unsigned long long)qp->max_results);
        return TS_ERR_CAPACITY;
    }
    if (total == 0) return TS_OK;
    TS_CUDA(pool_malloc((void **)&out->q, sizeof(uint32_t) * total, s));
    TS_CUDA(pool_malloc((void **)&out->e, sizeof(uint32_t) * total, s));
    TS_CUDA(pool_malloc((void **)&out->tin, sizeof(double) * total, s));
    TS_CUDA(pool_malloc((void **)&out->tout, sizeof(double) * total, s));
    b.out_q = out->q;
    b.out_e = out->e;
    b.out_tin = out->tin;
    b.out_tout = out->tout;
    c.rows = total;
    TS_CUDA(cudaEventRecord(ev_write.a, s));
    TS_CHECK(pipe_write(ix, w.reqdesc.as<ReqDesc>(), b, c, s));
    TS_CUDA(cudaEventRecord(ev_write.b, s));
    TS_CUDA(cudaMemcpyAsync(&st, b.status, 4, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    TS_CHECK(read_dev_status(st));
    out->stats.ms_write_pass = ev_write.ms();
    return TS_OK;
}

// The query columns of stationary points: x0 = x1 = x (likewise y, z), t0 = t_start, t1 = t_end.
__global__ void k_point_cols(const double *x, const double *y, const double *z, uint64_t n,
                             double ts, double te, double *cols)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double px = x[i], py = y[i], pz = z[i];
        cols[i] = px;
        cols[n + i] = py;
        cols[2 * n + i] = pz;
        cols[3 * n + i] = ts;
        cols[4 * n + i] = px;
        cols[5 * n + i] = py;
        cols[6 * n + i] = pz;
        cols[7 * n + i] = te;
    }
}

ts_status search_points(const Index *ix, const double *x, const double *y, const double *z,
                        uint64_t n, bool on_host, const ts_query_params *qp, cudaStream_t s,
                        SearchOut *out)
{
    TS_CHECK(check_query_params(qp));
    if (!(qp->t_start < qp->t_end)) {
        set_error("ts_search_points: the interval must have positive length");
        return TS_ERR_INVALID_ARG;
    }
    if (n && (!x || !y || !z)) {
        set_error("ts_search_points: NULL coordinate array");
        return TS_ERR_INVALID_ARG;
    }
    *out = SearchOut{};
    if (n == 0) return TS_OK;
    DevBuf pts, cols;
    const double *px = x, *py = y, *pz = z;
    if (on_host) {
        TS_CHECK(pts.alloc(sizeof(double) * 3 * n, s));
        double *d = pts.as<double>();
        TS_CUDA(cudaMemcpyAsync(d, x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        TS_CUDA(cudaMemcpyAsync(d + n, y, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        TS_CUDA(cudaMemcpyAsync(d + 2 * n, z, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        px = d;
        py = d + n;
        pz = d + 2 * n;
    }
    TS_CHECK(cols.alloc(sizeof(double) * 8 * n, s));
    k_point_cols<<<nblk(n), TPB, 0, s>>>(px, py, pz, n, qp->t_start, qp->t_end,
                                         cols.as<double>());
    TS_LAUNCHED();
    ts_segments q;
    memset(&q, 0, sizeof(q));
    const double *c = cols.as<double>();
    q.x0 = c; q.y0 = c + n; q.z0 = c + 2 * n; q.t0 = c + 3 * n;
    q.x1 = c + 4 * n; q.y1 = c + 5 * n; q.z1 = c + 6 * n; q.t1 = c + 7 * n;
    q.n = n;
    q.on_host = 0;
    return search_plain(ix, &q, qp, s, out);
}

ts_status schedule_only(const Index *ix, const ts_segments *q, const ts_query_params *qp,
                        cudaStream_t s, int32_t *sel, uint64_t *lo, uint64_t *hi)
{
    TS_CHECK(check_query_params(qp));
    if (!q || !sel || !lo || !hi) {
        set_error("ts_schedule: NULL argument");
        return TS_ERR_INVALID_ARG;
    }
    const uint64_t nq = q->n;
    if (nq == 0) return TS_OK;
    DevBuf qcopy;
    const double *cols[8];
    TS_CHECK(device_cols(q, s, qcopy, cols));
    PlainWork w;
    PipeBufs b;
    PipeCaps c;
    TS_CHECK(plain_prepare(ix, cols, nq, qp, s, w, b, c, false));
    uint32_t st = 0;
    if (ix->kind == TS_INDEX_SPATIAL) {
        // per query: number of z-runs and of candidates (sum of the runs' lengths)
        std::vector<uint32_t> off(nq + 1), ul(c.units), uh(c.units);
        TS_CUDA(cudaMemcpyAsync(off.data(), b.quoff, 4 * (nq + 1), cudaMemcpyDeviceToHost, s));
        if (c.units) {
            TS_CUDA(cudaMemcpyAsync(ul.data(), b.u_lo, 4 * c.units, cudaMemcpyDeviceToHost, s));
            TS_CUDA(cudaMemcpyAsync(uh.data(), b.u_hi, 4 * c.units, cudaMemcpyDeviceToHost, s));
        }
        TS_CUDA(cudaMemcpyAsync(&st, b.status, 4, cudaMemcpyDeviceToHost, s));
        TS_CUDA(cudaStreamSynchronize(s));
        TS_CHECK(read_dev_status(st));
        for (uint64_t i = 0; i < nq; i++) {
            sel[i] = SEL_GRID;
            lo[i] = off[i + 1] - off[i];
            uint64_t cand = 0;
            for (uint32_t u = off[i]; u < off[i + 1]; u++) cand += uh[u] - ul[u];
            hi[i] = cand;
        }
        return TS_OK;
    }
    std::vector<uint32_t> hs(nq), hl(nq), hh(nq);
    TS_CUDA(cudaMemcpyAsync(hs.data(), b.u_sel, 4 * nq, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(hl.data(), b.u_lo, 4 * nq, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(hh.data(), b.u_hi, 4 * nq, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(&st, b.status, 4, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    TS_CHECK(read_dev_status(st));
    for (uint64_t i = 0; i < nq; i++) {
        sel[i] = (int32_t)hs[i];
        lo[i] = hl[i];
        hi[i] = hh[i];
    }
    return TS_OK;
}

}  // namespace ts
