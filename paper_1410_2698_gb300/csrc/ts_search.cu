// ts_search.cu -- the search: query preparation, candidate schedule, query grouping, and the pair
// kernel with its count -> scan -> write result path.
//
// Paper mapping (Gowanlock & Casanova):
//   query preparation + schedule : the host-side schedule S of Sec. 4.2 and Sec. 4.3, here one
//                                  device thread per query segment (binary searches on the bin
//                                  prefix maximum replace the carried scan)
//   pair kernel                  : the compare() loop of Alg. 1-3; one warp sweeps the candidate
//                                  range of up to 32 queries (one per lane) instead of one thread
//                                  per query; results are counted, scanned and written at fixed
//                                  offsets instead of atomically appended to a fixed buffer.
//
// The pair test has two stages:
//   1. a conservative FP32 filter: time extents and MBBs rounded outward to FP32 (directed
//      rounding), the squared box distance accumulated rounding down; a pair is dropped only
//      when the lower bound of its separation exceeds d (with 1e-6 relative slack), so no pair
//      the FP64 test could accept is ever dropped;
//   2. the exact FP64 test on the survivors (the closed form of the interaction, evaluated
//      without FMA contraction so it reproduces the plain definition's rounding), compacted
//      32 at a time with ballot/popc so the FP64 pipe runs full warps.
#include <math.h>

#include <vector>

#include "ts_search.cuh"

namespace ts {

namespace {

constexpr int TPB = 256;
inline unsigned nblk(uint64_t n) { return (unsigned)((n + TPB - 1) / TPB ? (n + TPB - 1) / TPB : 1); }

// ---------------------------------------------------------------------------------------------
// PTX wrappers: mbarrier + 1-D bulk copy (TMA engine), globaltimer
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: gives up after ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && globaltimer_ns() - t0 > 2000000000ull) return false;
    }
}

// ---------------------------------------------------------------------------------------------
// exact FP64 interaction test (same operation order as the plain definition; no contraction)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double dmx(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double dmn(double a, double b) { return a < b ? a : b; }

struct Quad {
    double t_lo, T, a, b, c;
};

// Window and quadratic coefficients; false when the common window has no positive length.
__device__ __forceinline__ bool pair_quad(const QueryD &q, const SegD &e, double dd, Quad &o)
{
    double t_lo = dmx(q.w0, e.t0);
    double t_hi = dmn(q.w1, e.t1);
    if (!(t_lo < t_hi)) return false;
    double dq = t_lo - q.t0, de = t_lo - e.t0;
    double rx = (q.x0 + q.vx * dq) - (e.x0 + e.vx * de);
    double ry = (q.y0 + q.vy * dq) - (e.y0 + e.vy * de);
    double rz = (q.z0 + q.vz * dq) - (e.z0 + e.vz * de);
    double dvx = q.vx - e.vx, dvy = q.vy - e.vy, dvz = q.vz - e.vz;
    o.t_lo = t_lo;
    o.T = t_hi - t_lo;
    o.a = (dvx * dvx + dvy * dvy) + dvz * dvz;
    o.b = (rx * dvx + ry * dvy) + rz * dvz;
    o.c = ((rx * rx + ry * ry) + rz * rz) - dd;
    return true;
}

// Division-free hit decision: the minimum of a tau^2 + 2 b tau + c over [0, T] is <= 0.
__device__ __forceinline__ bool quad_hit(const Quad &k)
{
    if (k.a == 0.0) return k.c <= 0.0;
    if (k.b >= 0.0) return k.c <= 0.0;                       // minimum at tau = 0
    if (-k.b >= k.a * k.T) return (k.a * k.T + 2.0 * k.b) * k.T + k.c <= 0.0;  // at tau = T
    return k.b * k.b - k.a * k.c >= 0.0;                     // interior minimum
}

// Interval of a hit from the numerically stable root pair s/a, c/s.
__device__ __forceinline__ void quad_interval(const Quad &k, double *tin, double *tout)
{
    double lower, upper;
    if (k.a == 0.0) {
        lower = 0.0;
        upper = k.T;
    } else {
        double disc = k.b * k.b - k.a * k.c;
        if (disc < 0.0) disc = 0.0;  // only reachable within rounding of a tangency
        double sq = sqrt(disc);
        double s = -(k.b + copysign(sq, k.b));
        double r1, r2;
        if (s == 0.0) {
            r1 = 0.0;
            r2 = 0.0;
        } else {
            r1 = s / k.a;
            r2 = k.c / s;
        }
        lower = dmx(0.0, dmn(r1, r2));
        upper = dmn(k.T, dmx(r1, r2));
        if (upper < lower) upper = lower;  // only reachable within rounding of a tangency
    }
    *tin = k.t_lo + lower;
    *tout = k.t_lo + upper;
}

// Conservative FP32 filter (see file header).
__device__ __forceinline__ bool prefilter(const RecF &r, const float4 &qa, const float4 &qb,
                                          float d2u)
{
    bool t = (r.t0 < qb.w) && (r.t1 > qa.w);
    float gx = fmaxf(fmaxf(__fsub_rd(r.xmin, qb.x), __fsub_rd(qa.x, r.xmax)), 0.0f);
    float gy = fmaxf(fmaxf(__fsub_rd(r.ymin, qb.y), __fsub_rd(qa.y, r.ymax)), 0.0f);
    float gz = fmaxf(fmaxf(__fsub_rd(r.zmin, qb.z), __fsub_rd(qa.z, r.zmax)), 0.0f);
    float s2 = __fmaf_rd(gz, gz, __fmaf_rd(gy, gy, __fmul_rd(gx, gx)));
    return t && (s2 <= d2u);
}

// ---------------------------------------------------------------------------------------------
// query preparation and schedule (one thread per caller query)
// ---------------------------------------------------------------------------------------------
struct PrepParams {
    const double *f[8];
    uint64_t nq;
    int kind;
    double d, Ts, Te;
    // index
    uint64_t n;
    uint32_t m;
    double tmin, tmax;
    const double *bin_start, *bin_pmax;
    const uint32_t *bin_off;
    uint32_t v[3];
    double sub_lo[3], sub_w[3];
    const uint32_t *st_off[3];
    // outputs
    QueryD *qd;
    float4 *qf;
    uint32_t *qlo, *qhi, *qsel;
    uint64_t *keys;
    uint32_t *vals;
    unsigned long long *stats;
    uint32_t *status;
};

__device__ inline uint32_t first_pmax_above(const double *pmax, uint32_t m, double w0)
{
    uint32_t lo = 0, hi = m;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (pmax[mid] > w0) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// last bin with start < w1, or -1
__device__ inline int last_start_below(const double *bs, uint32_t m, double w1)
{
    uint32_t lo = 0, hi = m;  // first j with bs[j] >= w1
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (bs[mid] >= w1) hi = mid; else lo = mid + 1;
    }
    return (int)lo - 1;
}

__global__ void k_qprep(PrepParams P)
{
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool in = i < P.nq;
    bool valid = false, subbin = false;
    if (in) {
        double v[8];
        bool fin = true;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            v[k] = P.f[k][i];
            fin = fin && isfinite(v[k]);
        }
        if (!fin || !(v[7] > v[3])) atomicOr(P.status, DEV_ERR_INVALID);
        double dt = v[7] - v[3];
        QueryD q;
        q.x0 = v[0]; q.y0 = v[1]; q.z0 = v[2]; q.t0 = v[3];
        q.vx = (v[4] - v[0]) / dt;
        q.vy = (v[5] - v[1]) / dt;
        q.vz = (v[6] - v[2]) / dt;
        q.w0 = dmx(v[3], P.Ts);
        q.w1 = dmn(v[7], P.Te);
        q.pad = 0.0;
        valid = fin && (v[7] > v[3]) && (q.w0 < q.w1);
        P.qd[i] = q;
        double mn[3], mx[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            mn[d] = v[d] < v[4 + d] ? v[d] : v[4 + d];
            mx[d] = v[d] < v[4 + d] ? v[4 + d] : v[d];
        }
        P.qf[2 * i] = make_float4(__double2float_rd(mn[0]), __double2float_rd(mn[1]),
                                  __double2float_rd(mn[2]), __double2float_rd(q.w0));
        P.qf[2 * i + 1] = make_float4(__double2float_ru(mx[0]), __double2float_ru(mx[1]),
                                      __double2float_ru(mx[2]), __double2float_ru(q.w1));
        uint32_t sel = SEL_T, lo = 0, hi = 0, j = 0;
        if (valid) {
            if (P.kind == TS_INDEX_BRUTE) {
                lo = 0;
                hi = (uint32_t)P.n;
            } else {
                // temporal range (Sec. 4.2 schedule)
                uint32_t jl = first_pmax_above(P.bin_pmax, P.m, q.w0);
                int jh = last_start_below(P.bin_start, P.m, q.w1);
                bool any = (int)jl <= jh;
                if (any) {
                    lo = P.bin_off[jl];
                    hi = P.bin_off[jh + 1];
                }
                if (any && P.kind == TS_INDEX_SPATIOTEMPORAL) {
                    // dimension whose d-expanded extent meets one subbin (or none) with the
                    // fewest ids over the bins jl..jh (Sec. 4.3 schedule)
                    long long best = -1;
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        int vv = (int)P.v[d];
                        int pa = part_of(mn[d] - P.d, P.sub_lo[d], P.sub_w[d], vv);
                        int pb = part_of(mx[d] + P.d, P.sub_lo[d], P.sub_w[d], vv);
                        int ja = pa < 0 ? 0 : pa, jb = pb;
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
                            j = jb < ja ? 0u : (uint32_t)ja;
                        }
                    }
                    subbin = best >= 0;
                }
            }
        }
        P.qlo[i] = lo;
        P.qhi[i] = hi;
        P.qsel[i] = sel;
        uint64_t key = ~0ull;
        if (valid) {
            double span = P.tmax - P.tmin;
            double u = span > 0.0 ? (q.w0 - P.tmin) / span : 0.0;
            u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
            uint32_t qt = (uint32_t)(u * 4294967295.0);
            uint32_t gk = (sel << 28) | (j & 0x0fffffffu);
            key = ((uint64_t)gk << 32) | qt;
        }
        P.keys[i] = key;
        P.vals[i] = (uint32_t)i;
    }
    unsigned vm = __ballot_sync(0xffffffffu, valid);
    unsigned sm = __ballot_sync(0xffffffffu, subbin);
    if ((threadIdx.x & 31) == 0) {
        if (vm) atomicAdd(&P.stats[ST_QSEGS], (unsigned long long)__popc(vm));
        if (sm) atomicAdd(&P.stats[ST_SUBBIN], (unsigned long long)__popc(sm));
    }
}

// ---------------------------------------------------------------------------------------------
// grouping: runs of equal group key in sorted order, cut into groups of <= 32 queries
// ---------------------------------------------------------------------------------------------
__device__ inline uint32_t gk_of(uint64_t key) { return (uint32_t)(key >> 32); }

__global__ void k_group_mark(const uint64_t *keys, uint64_t nq, const unsigned long long *stats,
                             uint32_t *flags)
{
    uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nq) return;
    uint64_t nvalid = stats[ST_QSEGS];
    if (p >= nvalid) {
        flags[p] = 0;
        return;
    }
    uint32_t gk = gk_of(keys[p]);
    uint64_t lo = 0, hi = p;  // first position of this run
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (gk_of(keys[mid]) < gk) lo = mid + 1; else hi = mid;
    }
    flags[p] = ((p - lo) % 32u) == 0 ? 1u : 0u;
}

__global__ void k_group_fill(const uint64_t *keys, const uint32_t *vals, uint64_t nq,
                             const unsigned long long *stats, const uint32_t *flags,
                             const uint32_t *gid, const uint32_t *qlo, const uint32_t *qhi,
                             Group *groups, uint32_t *ntiles)
{
    uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nq || !flags[p]) return;
    uint64_t nvalid = stats[ST_QSEGS];
    uint32_t gk = gk_of(keys[p]);
    uint64_t lo = p, hi = nvalid;  // end of this run
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (gk_of(keys[mid]) <= gk) lo = mid + 1; else hi = mid;
    }
    uint32_t cnt = (uint32_t)((lo - p) < 32 ? (lo - p) : 32);
    uint32_t ulo = 0xffffffffu, uhi = 0;
    for (uint32_t k = 0; k < cnt; k++) {
        uint32_t ci = vals[p + k];
        if (qhi[ci] > qlo[ci]) {
            ulo = min(ulo, qlo[ci]);
            uhi = max(uhi, qhi[ci]);
        }
    }
    if (uhi <= ulo) {
        ulo = 0;
        uhi = 0;
    }
    Group g;
    g.first = (uint32_t)p;
    g.count = cnt;
    g.sel = gk >> 28;
    g.lo = ulo;
    g.hi = uhi;
    g.pad[0] = g.pad[1] = g.pad[2] = 0;
    uint32_t id = gid[p];
    groups[id] = g;
    ntiles[id] = (uhi - ulo + PK_TILE - 1) / PK_TILE;
}

__global__ void k_hdr(const unsigned long long *stats_in, const uint32_t *gid, const uint64_t *tile_base,
                      uint64_t nq, uint32_t *hdr, unsigned long long *stats)
{
    uint32_t ng = gid[nq];
    uint64_t nt = tile_base[nq];
    hdr[HDR_NVALID] = (uint32_t)stats_in[ST_QSEGS];
    hdr[HDR_NGROUPS] = ng;
    hdr[HDR_NTILES_LO] = (uint32_t)nt;
    hdr[HDR_NTILES_HI] = (uint32_t)(nt >> 32);
    stats[ST_GROUPS] = ng;
    stats[ST_TILES] = nt;
}

// ---------------------------------------------------------------------------------------------
// pair kernel
// ---------------------------------------------------------------------------------------------
struct __align__(16) WarpSmem {
    RecF stage[2][PK_CH];
    QueryD qd[32];
    uint32_t qorig[32];
    uint32_t queue[64];
    unsigned long long bar[2];
    uint32_t pad[2];
};

enum { PASS_COUNT = 0, PASS_WRITE = 1 };

__device__ __forceinline__ uint32_t find_group(const uint64_t *base, uint32_t ng, uint64_t t)
{
    uint32_t lo = 0, hi = ng;  // first g with base[g] > t, minus one
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (base[mid] <= t) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

template <int PASS>
__global__ void __launch_bounds__(PK_THREADS, 2) k_pair(PairParams P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    WarpSmem &W = reinterpret_cast<WarpSmem *>(smem_raw)[wid];
    const unsigned FULL = 0xffffffffu;
    const uint32_t lt_mask = (1u << lane) - 1u;

    if (lane == 0) {
        mbar_init(&W.bar[0], 1);
        mbar_init(&W.bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool abort = false;

    const uint32_t ngroups = P.hdr[HDR_NGROUPS];
    const uint64_t ntiles = (uint64_t)P.hdr[HDR_NTILES_LO] | ((uint64_t)P.hdr[HDR_NTILES_HI] << 32);
    unsigned long long acc_tests = 0, acc_exact = 0, acc_hits = 0;

    while (!abort) {
        uint64_t t = 0;
        if (lane == 0) t = atomicAdd(P.tile_counter, 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= ntiles) break;
        const uint32_t g = find_group(P.tile_base, ngroups, t);
        const Group G = P.groups[g];
        const uint32_t s0 = G.lo + (uint32_t)(t - P.tile_base[g]) * PK_TILE;
        const uint32_t s1 = min(G.hi, s0 + PK_TILE);
        const RecF *recs = P.rec[G.sel];
        const uint32_t *ids = P.ids[G.sel];

        // this lane's query
        const bool act = (uint32_t)lane < G.count;
        float4 qa = make_float4(0.f, 0.f, 0.f, 0.f), qb = qa;
        uint32_t qlo = 0, qhi = 0;
        if (act) {
            uint32_t ci = P.qval[G.first + lane];
            qa = P.qf[2 * (uint64_t)ci];
            qb = P.qf[2 * (uint64_t)ci + 1];
            qlo = P.qlo[ci];
            qhi = P.qhi[ci];
            W.qd[lane] = P.qd[ci];
            W.qorig[lane] = ci;
        }
        if (PASS == PASS_COUNT) {
            uint32_t a = max(qlo, s0), b = min(qhi, s1);
            acc_tests += (act && b > a) ? (b - a) : 0u;
        }
        __syncwarp();

        const uint32_t nrec = s1 - s0;
        const uint32_t nch = (nrec + PK_CH - 1) / PK_CH;
        if (lane == 0) {
            for (uint32_t k = 0; k < 2 && k < nch; k++) {
                uint32_t cs = s0 + k * PK_CH, cn = min((uint32_t)PK_CH, s1 - cs);
                mbar_arrive_tx(&W.bar[k], cn * (uint32_t)sizeof(RecF));
                bulk_g2s(&W.stage[k][0], recs + cs, cn * (uint32_t)sizeof(RecF), &W.bar[k]);
            }
        }
        pending[0] = nch > 0;
        pending[1] = nch > 1;

        uint32_t qn = 0, hits = 0;
        const uint64_t wbase = PASS == PASS_WRITE ? P.tile_off[t] : 0;
        const uint64_t wend = PASS == PASS_WRITE ? P.tile_off[t + 1] : 0;

        auto flush = [&](uint32_t k) {
            uint32_t item = (uint32_t)lane < k ? W.queue[lane] : 0u;
            __syncwarp();
            if (qn > k && (uint32_t)lane < qn - k) W.queue[lane] = W.queue[k + lane];
            __syncwarp();
            bool h = false;
            double tin = 0.0, tout = 0.0;
            uint32_t qlane = item >> 27, eid = 0;
            if ((uint32_t)lane < k) {
                uint32_t pos = s0 + (item & 0x07ffffffu);
                eid = ids ? ids[pos] : pos;
                const SegD e = P.seg[eid];
                const QueryD q = W.qd[qlane];
                Quad qd;
                if (pair_quad(q, e, P.dd, qd) && quad_hit(qd)) {
                    h = true;
                    if (PASS == PASS_WRITE) quad_interval(qd, &tin, &tout);
                }
            }
            unsigned hm = __ballot_sync(FULL, h);
            if (PASS == PASS_WRITE && h) {
                uint64_t o = wbase + hits + __popc(hm & lt_mask);
                if (o < wend) {
                    P.out_q[o] = W.qorig[qlane];
                    P.out_e[o] = P.orig[eid];
                    P.out_tin[o] = tin;
                    P.out_tout[o] = tout;
                }
            }
            hits += __popc(hm);
            acc_exact += k;
            qn -= k;
        };

        for (uint32_t k = 0; k < nch && !abort; k++) {
            const int st = k & 1;
            if (!mbar_wait_bounded(&W.bar[st], parity[st])) {
                abort = true;
                break;
            }
            parity[st] ^= 1u;
            pending[st] = false;
            const uint32_t cs = s0 + k * PK_CH;
            const uint32_t cn = min((uint32_t)PK_CH, s1 - cs);
            const RecF *buf = &W.stage[st][0];
            for (uint32_t j = 0; j < cn; j++) {
                const RecF r = buf[j];
                const uint32_t pos = cs + j;
                const bool pass = act && pos >= qlo && pos < qhi && prefilter(r, qa, qb, P.d2u);
                const unsigned m = __ballot_sync(FULL, pass);
                if (m) {
                    if (pass) W.queue[qn + __popc(m & lt_mask)] = ((uint32_t)lane << 27) | (pos - s0);
                    qn += __popc(m);
                    if (qn >= 32) {
                        __syncwarp();
                        flush(32);
                    }
                }
            }
            __syncwarp();
            if (k + 2 < nch) {
                if (lane == 0) {
                    uint32_t ns = s0 + (k + 2) * PK_CH, nn = min((uint32_t)PK_CH, s1 - ns);
                    mbar_arrive_tx(&W.bar[st], nn * (uint32_t)sizeof(RecF));
                    bulk_g2s(&W.stage[st][0], recs + ns, nn * (uint32_t)sizeof(RecF), &W.bar[st]);
                }
                pending[st] = true;
            }
        }
        if (abort) break;
        if (qn) {
            __syncwarp();
            flush(qn);
        }
        if (PASS == PASS_COUNT) {
            if (lane == 0) P.tile_hits[t] = hits;
            acc_hits += hits;
        } else {
            if (lane == 0 && wbase + hits != wend) atomicOr(P.status, DEV_ERR_INTERNAL);
        }
        __syncwarp();
    }
    if (abort) {
        if (lane == 0) atomicOr(P.status, DEV_ERR_TIMEOUT);
        // let copies still in flight land before the shared memory is released
        for (int st = 0; st < 2; st++)
            if (pending[st]) mbar_wait_bounded(&W.bar[st], parity[st]);
    }
    if (PASS == PASS_COUNT) {
        for (int o = 16; o; o >>= 1) acc_tests += __shfl_xor_sync(FULL, acc_tests, o);
        if (lane == 0) {
            atomicAdd(&P.stats[ST_TESTS], acc_tests);
            atomicAdd(&P.stats[ST_EXACT], acc_exact);
            atomicAdd(&P.stats[ST_HITS], acc_hits);
        }
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

}  // namespace

// ---------------------------------------------------------------------------------------------
// host orchestration of one plain search
// ---------------------------------------------------------------------------------------------

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
static float float_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

static ts_status read_dev_status(uint32_t st)
{
    if (st & DEV_ERR_INVALID) {
        set_error("invalid query segment (NaN/Inf or t_end <= t_start)");
        return TS_ERR_INVALID_ARG;
    }
    if (st & DEV_ERR_TIMEOUT) {
        set_error("a bounded device wait ran out (TMA copy did not complete)");
        return TS_ERR_TIMEOUT;
    }
    if (st) {
        set_error("search: device status 0x%x", st);
        return TS_ERR_INTERNAL;
    }
    return TS_OK;
}

// Runs query preparation and grouping; fills the work buffers. Returns the device pointers the
// pair kernel needs through P (outputs left unset).
static ts_status prepare(const Index *ix, const double *const cols[8], uint64_t nq,
                         const ts_query_params *qp, cudaStream_t s, SearchWork &w, PairParams &P)
{
    TS_CHECK(w.qd.alloc(sizeof(QueryD) * nq, s));
    TS_CHECK(w.qf.alloc(sizeof(float4) * 2 * nq, s));
    TS_CHECK(w.qlo.alloc(sizeof(uint32_t) * nq, s));
    TS_CHECK(w.qhi.alloc(sizeof(uint32_t) * nq, s));
    TS_CHECK(w.qsel.alloc(sizeof(uint32_t) * nq, s));
    TS_CHECK(w.keys.alloc(sizeof(uint64_t) * nq, s));
    TS_CHECK(w.vals.alloc(sizeof(uint32_t) * nq, s));
    TS_CHECK(w.flags.alloc(sizeof(uint32_t) * nq, s));
    TS_CHECK(w.gid.alloc(sizeof(uint32_t) * (nq + 1), s));
    TS_CHECK(w.groups.alloc(sizeof(Group) * nq, s));
    TS_CHECK(w.ntiles.alloc(sizeof(uint32_t) * nq, s));
    TS_CHECK(w.tile_base.alloc(sizeof(uint64_t) * (nq + 1), s));
    TS_CHECK(w.hdr.alloc(sizeof(uint32_t) * HDR_N, s));
    TS_CHECK(w.stats.alloc(sizeof(unsigned long long) * ST_NSLOTS, s));
    TS_CHECK(w.status.alloc(sizeof(uint32_t), s));
    TS_CHECK(w.counters.alloc(sizeof(uint32_t) * 2, s));
    TS_CUDA(cudaMemsetAsync(w.stats.p, 0, sizeof(unsigned long long) * ST_NSLOTS, s));
    TS_CUDA(cudaMemsetAsync(w.status.p, 0, sizeof(uint32_t), s));
    TS_CUDA(cudaMemsetAsync(w.counters.p, 0, sizeof(uint32_t) * 2, s));
    TS_CUDA(cudaMemsetAsync(w.ntiles.p, 0, sizeof(uint32_t) * nq, s));

    PrepParams pp;
    for (int k = 0; k < 8; k++) pp.f[k] = cols[k];
    pp.nq = nq;
    pp.kind = ix->kind;
    pp.d = qp->d;
    pp.Ts = qp->t_start;
    pp.Te = qp->t_end;
    pp.n = ix->n;
    pp.m = ix->m;
    pp.tmin = ix->tmin;
    pp.tmax = ix->tmax;
    pp.bin_start = ix->bin_start;
    pp.bin_pmax = ix->bin_pmax;
    pp.bin_off = ix->bin_off;
    for (int d = 0; d < 3; d++) {
        pp.v[d] = ix->v[d];
        pp.sub_lo[d] = ix->sub_lo[d];
        pp.sub_w[d] = ix->sub_w[d];
        pp.st_off[d] = ix->st_off[d];
    }
    pp.qd = w.qd.as<QueryD>();
    pp.qf = w.qf.as<float4>();
    pp.qlo = w.qlo.as<uint32_t>();
    pp.qhi = w.qhi.as<uint32_t>();
    pp.qsel = w.qsel.as<uint32_t>();
    pp.keys = w.keys.as<uint64_t>();
    pp.vals = w.vals.as<uint32_t>();
    pp.stats = w.stats.as<unsigned long long>();
    pp.status = w.status.as<uint32_t>();
    k_qprep<<<nblk(nq), TPB, 0, s>>>(pp);
    TS_LAUNCHED();

    TS_CHECK(radix_sort_u64(w.keys.as<uint64_t>(), w.vals.as<uint32_t>(), nq, 64, s));
    k_group_mark<<<nblk(nq), TPB, 0, s>>>(w.keys.as<uint64_t>(), nq,
                                          w.stats.as<unsigned long long>(), w.flags.as<uint32_t>());
    TS_LAUNCHED();
    TS_CHECK(scan_u32(w.flags.as<uint32_t>(), w.gid.as<uint32_t>(), nq, w.status.as<uint32_t>(), s));
    k_group_fill<<<nblk(nq), TPB, 0, s>>>(w.keys.as<uint64_t>(), w.vals.as<uint32_t>(), nq,
                                          w.stats.as<unsigned long long>(), w.flags.as<uint32_t>(),
                                          w.gid.as<uint32_t>(), w.qlo.as<uint32_t>(),
                                          w.qhi.as<uint32_t>(), w.groups.as<Group>(),
                                          w.ntiles.as<uint32_t>());
    TS_LAUNCHED();
    TS_CHECK(scan_u32_to_u64(w.ntiles.as<uint32_t>(), w.tile_base.as<uint64_t>(), nq, s));
    k_hdr<<<1, 1, 0, s>>>(w.stats.as<unsigned long long>(), w.gid.as<uint32_t>(),
                          w.tile_base.as<uint64_t>(), nq, w.hdr.as<uint32_t>(),
                          w.stats.as<unsigned long long>());
    TS_LAUNCHED();

    P = PairParams{};
    P.groups = w.groups.as<Group>();
    P.tile_base = w.tile_base.as<uint64_t>();
    P.hdr = w.hdr.as<uint32_t>();
    P.qval = w.vals.as<uint32_t>();
    P.qd = w.qd.as<QueryD>();
    P.qf = w.qf.as<float4>();
    P.qlo = w.qlo.as<uint32_t>();
    P.qhi = w.qhi.as<uint32_t>();
    for (int k = 0; k < 3; k++) {
        P.rec[k] = ix->st_rec[k];
        P.ids[k] = ix->st_ids[k];
    }
    P.rec[SEL_T] = ix->rec;
    P.ids[SEL_T] = nullptr;
    P.rec[SEL_GRID] = ix->ga_rec;
    P.ids[SEL_GRID] = ix->ga;
    P.seg = ix->seg;
    P.orig = ix->orig;
    P.dd = qp->d * qp->d;
    P.d2u = float_up(P.dd * (1.0 + 1e-6));
    P.stats = w.stats.as<unsigned long long>();
    P.status = w.status.as<uint32_t>();
    return TS_OK;
}

static ts_status device_cols(const ts_segments *q, cudaStream_t s, DevBuf &copy, const double *cols[8])
{
    const double *src[8] = {q->x0, q->y0, q->z0, q->t0, q->x1, q->y1, q->z1, q->t1};
    for (int k = 0; k < 8; k++)
        if (!src[k]) {
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

static ts_status check_query_params(const ts_query_params *qp)
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
    if (ix->kind == TS_INDEX_SPATIAL) {
        set_error("the spatial grid search runs through ts_search_spatial");
        return TS_ERR_INVALID_ARG;
    }
    *out = SearchOut{};
    const uint64_t nq = q->n;
    out->stats.n_queries = nq;
    if (nq == 0) return TS_OK;
    DevBuf qcopy;
    const double *cols[8];
    TS_CHECK(device_cols(q, s, qcopy, cols));
    SearchWork w;
    PairParams P;
    TS_CHECK(prepare(ix, cols, nq, qp, s, w, P));

    uint32_t hdr[HDR_N];
    uint32_t st = 0;
    TS_CUDA(cudaMemcpyAsync(hdr, w.hdr.p, sizeof(hdr), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(&st, w.status.p, 4, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    TS_CHECK(read_dev_status(st));
    const uint64_t ntiles = (uint64_t)hdr[HDR_NTILES_LO] | ((uint64_t)hdr[HDR_NTILES_HI] << 32);

    int blocks = 0;
    TS_CHECK(pair_grid(&blocks));
    const size_t smem = sizeof(WarpSmem) * PK_WARPS;
    TS_CHECK(w.tile_hits.alloc(sizeof(uint32_t) * (ntiles ? ntiles : 1), s));
    TS_CHECK(w.tile_off.alloc(sizeof(uint64_t) * (ntiles + 1), s));
    P.tile_hits = w.tile_hits.as<uint32_t>();
    P.tile_counter = w.counters.as<uint32_t>();
    EventPair ev_count, ev_write;
    TS_CHECK(ev_count.create());
    TS_CHECK(ev_write.create());
    TS_CUDA(cudaEventRecord(ev_count.a, s));
    if (ntiles) {
        k_pair<PASS_COUNT><<<blocks, PK_THREADS, smem, s>>>(P);
        TS_LAUNCHED();
    }
    TS_CUDA(cudaEventRecord(ev_count.b, s));
    TS_CHECK(scan_u32_to_u64(w.tile_hits.as<uint32_t>(), w.tile_off.as<uint64_t>(), ntiles, s));
    uint64_t total = 0;
    unsigned long long hst[ST_NSLOTS];
    TS_CUDA(cudaMemcpyAsync(&total, w.tile_off.as<uint64_t>() + ntiles, 8, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(hst, w.stats.p, sizeof(hst), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(&st, w.status.p, 4, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    TS_CHECK(read_dev_status(st));
    out->count = total;
    out->stats.n_qsegs = hst[ST_QSEGS];
    out->stats.n_tests = hst[ST_TESTS];
    out->stats.n_exact = hst[ST_EXACT];
    out->stats.n_hits = hst[ST_HITS];
    out->stats.n_tiles = hst[ST_TILES];
    out->stats.n_groups = hst[ST_GROUPS];
    out->stats.n_subbin = hst[ST_SUBBIN];
    out->stats.ms_count_pass = ev_count.ms();
    if (hst[ST_HITS] != total) {
        set_error("hit count mismatch (%llu vs %llu)", (unsigned long long)hst[ST_HITS],
                  (unsigned long long)total);
        return TS_ERR_INTERNAL;
    }
    if (qp->max_results && total > qp->max_results) {
        set_error("%llu result rows exceed max_results %llu", (unsigned long long)total,
                  (unsigned long long)qp->max_results);
        return TS_ERR_CAPACITY;
    }
    if (total == 0) return TS_OK;
    TS_CUDA(cudaMallocAsync((void **)&out->q, sizeof(uint32_t) * total, s));
    TS_CUDA(cudaMallocAsync((void **)&out->e, sizeof(uint32_t) * total, s));
    TS_CUDA(cudaMallocAsync((void **)&out->tin, sizeof(double) * total, s));
    TS_CUDA(cudaMallocAsync((void **)&out->tout, sizeof(double) * total, s));
    P.tile_off = w.tile_off.as<uint64_t>();
    P.out_q = out->q;
    P.out_e = out->e;
    P.out_tin = out->tin;
    P.out_tout = out->tout;
    P.tile_counter = w.counters.as<uint32_t>() + 1;
    TS_CUDA(cudaEventRecord(ev_write.a, s));
    k_pair<PASS_WRITE><<<blocks, PK_THREADS, smem, s>>>(P);
    TS_LAUNCHED();
    TS_CUDA(cudaEventRecord(ev_write.b, s));
    TS_CUDA(cudaMemcpyAsync(&st, w.status.p, 4, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    TS_CHECK(read_dev_status(st));
    out->stats.ms_write_pass = ev_write.ms();
    return TS_OK;
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
    if (ix->kind == TS_INDEX_SPATIAL) {
        set_error("ts_schedule: the spatial grid schedule runs through ts_search_spatial");
        return TS_ERR_INVALID_ARG;
    }
    DevBuf qcopy;
    const double *cols[8];
    TS_CHECK(device_cols(q, s, qcopy, cols));
    SearchWork w;
    PairParams P;
    TS_CHECK(prepare(ix, cols, nq, qp, s, w, P));
    std::vector<uint32_t> hs(nq), hl(nq), hh(nq);
    uint32_t st = 0;
    TS_CUDA(cudaMemcpyAsync(hs.data(), w.qsel.p, 4 * nq, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(hl.data(), w.qlo.p, 4 * nq, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(hh.data(), w.qhi.p, 4 * nq, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(&st, w.status.p, 4, cudaMemcpyDeviceToHost, s));
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
