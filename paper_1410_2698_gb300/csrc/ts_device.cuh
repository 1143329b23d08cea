// ts_device.cuh -- device helpers of the pair test: PTX wrappers for the bulk-copy engine and
// mbarriers, the exact FP64 interaction test and the conservative FP32 filter.
#pragma once

#include "ts_internal.cuh"

namespace ts {

// ---------------------------------------------------------------------------------------------
// PTX wrappers: mbarrier + 1-D bulk copy (TMA engine), globaltimer
// ---------------------------------------------------------------------------------------------
static __device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

static __device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

static __device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

static __device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

static __device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

static __device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
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

static __device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Limit of every bounded wait on a copy: 2 s of wall time.
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

// Bounded wait on an mbarrier phase: gives up (false) after limit_ns of wall time.
static __device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity,
                                                         uint64_t limit_ns = WAIT_LIMIT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// ---------------------------------------------------------------------------------------------
// exact FP64 interaction test
// ---------------------------------------------------------------------------------------------
// Every multiply-add of the test is an explicit fma() (one FP64 instruction and one rounding; the
// rest of the library is compiled without contraction, so the rounding of each step is exactly
// the one written here). The test differs from the plain definition's evaluation by a few
// rounding errors, which only matters for pairs whose minimum separation is within rounding of d.
static __device__ __forceinline__ double dmx(double a, double b) { return a > b ? a : b; }
static __device__ __forceinline__ double dmn(double a, double b) { return a < b ? a : b; }

// The bit pattern of an FP64 value, read through a register move the compiler cannot see into:
// integer tests on the pattern (signs, zeros, orders, below) then stay integer instructions,
// where a plain reinterpretation lets the compiler turn some of them back into FP64 compares and
// absolute values.
static __device__ __forceinline__ long long dbits(double x)
{
    long long v;
    asm("mov.b64 %0, %1;" : "=l"(v) : "d"(x));
    return v;
}

struct Quad {
    double t_lo, T, a, b, c;
};

// Window and quadratic coefficients; false when the common window has no positive length.
// r0 = p_q(t_lo) - p_l(t_lo), dv = v_q - v_l, a = dv.dv, b = r0.dv, c = r0.r0 - d^2.
// When the four window bounds have their sign bits clear (non-negative times, the usual case) the
// window is found on the integer pipe: non-negative doubles order as their bit patterns.
//
// t_lo is the later of the two starts (the query's clipped w0, where its record holds its
// position, or the entry's t0), so one of the two positions at t_lo is a start point as stored
// and only the other segment is advanced, by dt = t_lo - its own start: s r0 = (p_adv + v_adv dt)
// - p_start, where s = +1 when the query is the segment advanced and -1 when the entry is. With
// dv taken in the same orientation (s dv = v_adv - v_start), b = (s r0).(s dv) needs no sign
// correction, and a and c do not depend on s.
static __device__ __forceinline__ bool pair_quad(const QueryD &q, const SegD &e, Quad &o)
{
    double t_lo, t_hi;
    bool adv_q;  // the entry starts at t_lo (or both do): advance the query
    const long long a0 = dbits(q.w0), b0 = dbits(e.t0);
    const long long a1 = dbits(q.w1), b1 = dbits(e.t1);
    if ((a0 | b0 | a1 | b1) >= 0) {
        adv_q = b0 >= a0;
        const long long lo = adv_q ? b0 : a0, hi = a1 < b1 ? a1 : b1;
        if (!(lo < hi)) return false;
        t_lo = __longlong_as_double(lo);
        t_hi = __longlong_as_double(hi);
    } else {
        adv_q = e.t0 >= q.w0;
        t_lo = adv_q ? e.t0 : q.w0;
        t_hi = dmn(q.w1, e.t1);
        if (!(t_lo < t_hi)) return false;
    }
    const double dt = t_lo - (adv_q ? q.w0 : e.t0);
    const double rx = fma(adv_q ? q.vx : e.vx, dt, adv_q ? q.xw : e.x0) - (adv_q ? e.x0 : q.xw);
    const double ry = fma(adv_q ? q.vy : e.vy, dt, adv_q ? q.yw : e.y0) - (adv_q ? e.y0 : q.yw);
    const double rz = fma(adv_q ? q.vz : e.vz, dt, adv_q ? q.zw : e.z0) - (adv_q ? e.z0 : q.zw);
    const double dvx = (adv_q ? q.vx : e.vx) - (adv_q ? e.vx : q.vx);
    const double dvy = (adv_q ? q.vy : e.vy) - (adv_q ? e.vy : q.vy);
    const double dvz = (adv_q ? q.vz : e.vz) - (adv_q ? e.vz : q.vz);
    o.t_lo = t_lo;
    o.T = t_hi - t_lo;
    o.a = fma(dvz, dvz, fma(dvy, dvy, dvx * dvx));
    o.b = fma(rz, dvz, fma(ry, dvy, rx * dvx));
    o.c = fma(rz, rz, fma(ry, ry, fma(rx, rx, q.ndd)));
    return true;
}

// Sign and order tests of FP64 values made on their bit patterns, so that they run on the integer
// pipe instead of the FP64 pipe (on GB300 an FP64 instruction costs as much pipe time as 32 integer
// ones). For values that are not NaN; -0.0 and +0.0 compare equal, as in IEEE arithmetic.
// x < 0 (sign bit set and not -0.0)
static __device__ __forceinline__ bool neg(double x)
{
    const long long v = dbits(x);
    return v < 0 && (v << 1) != 0;
}
// x <= 0 (a set sign bit as a signed integer is negative; +0.0 is 0)
static __device__ __forceinline__ bool nonpos(double x) { return dbits(x) <= 0; }
// x == 0
static __device__ __forceinline__ bool zero(double x) { return (dbits(x) << 1) == 0; }
// |x| < |y|: the magnitudes order as their bit patterns with the sign bit shifted out (a shift,
// not a mask: the compiler reads a masked-off sign bit as an FP64 absolute value)
static __device__ __forceinline__ bool mag_lt(double x, double y)
{
    return ((unsigned long long)dbits(x) << 1) < ((unsigned long long)dbits(y) << 1);
}

// |x| within [2^-1000, 2^1000) (its biased exponent, sign ignored): the range where the refined
// estimates below are accurate (no subnormal estimate, no overflow of x * y).
static __device__ __forceinline__ bool nr_range(double x)
{
    const uint32_t ex = ((uint32_t)__double2hiint(x) >> 20) & 0x7ffu;
    return ex - 23u < 2000u;
}

// 1/x by Newton-Raphson from the hardware estimate (rcp.approx.ftz.f64, about 20 good bits): one
// second-order step y + y e with e = 1 - x y squares the estimate's relative error, to about
// 2^-40 (measured 2^-39.9 over the range): a thousandth of the 1e-9 interval tolerance, for two
// FP64 instructions. For x in the nr_range.
static __device__ __forceinline__ double rcp_nr(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// sqrt(x) by Newton-Raphson from the hardware estimate y of 1/sqrt(x) (rsqrt.approx.ftz.f64):
// g = x y ~ sqrt(x), then one Newton correction of g with the residual x - g^2 and h = y / 2 ~
// 1/(2 sqrt(x)). With y of relative error eps, the result's is about 1.5 eps^2 (measured 2^-39.5
// over the range). For x in the nr_range (the estimate is then a normal number, and halving it is
// a decrement of its exponent, on the integer pipe).
static __device__ __forceinline__ double sqrt_nr(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double g = x * y, h = __longlong_as_double(dbits(y) - (1ll << 52));
    return fma(fma(-g, g, x), h, g);
}

// Hit decision and, when `interval`, the hit interval [*tin, *tout].
//
// The decision is division-free: the minimum of a tau^2 + 2 b tau + c over [0, T] is <= 0 (a >= 0,
// T > 0). Its branch tests are sign and magnitude tests on the integer pipe: a is a sum of
// squares, and -b and aT are compared only when b < 0. The discriminant disc = b^2 - a c decides
// an interior minimum and gives the roots, so it is computed once, before the branches (a warp
// whose lanes take different branches issues every branch's instructions, so a value two
// branches need is cheapest computed once for all lanes).
//
// The interval comes from the numerically stable root pair s/a, c/s (s = -(b + sign(b)
// sqrt(disc))). The square root and the two quotients come from the refined estimates above
// (relative error about 2^-40 each, so a few 1e-12 of the roots: far inside the 1e-9 interval
// tolerance); values outside their range take the library's sqrt and division. The code carries
// t = -s and writes the roots as (-t)/a and (-c)/t, so that the negations are operand modifiers
// of the multiplies rather than FP64 instructions of their own. The roots need no comparison of
// their values: with s of the sign opposite to b's sign bit, s/a is the smaller root when b's
// sign bit is clear and the larger when it is set (c/s is the other), and every clamp compares a
// value with 0 or two non-negative values, which the integer pipe does on the bit patterns.
static __device__ __forceinline__ bool quad_solve(const Quad &k, bool interval, double *tin,
                                                  double *tout)
{
    double disc = fma(k.b, k.b, -(k.a * k.c));
    bool hit;
    if (zero(k.a) || !neg(k.b)) {
        hit = nonpos(k.c);                                         // minimum at tau = 0
    } else {
        const double aT = k.a * k.T;
        if (!mag_lt(k.b, aT))
            hit = nonpos(fma(fma(2.0, k.b, aT), k.T, k.c));        // at tau = T (-b >= aT)
        else
            hit = !neg(disc);                                      // interior minimum
    }
    if (!hit || !interval) return hit;
    double lower, upper;
    if (zero(k.a)) {
        lower = 0.0;
        upper = k.T;
    } else {
        if (neg(disc)) disc = 0.0;  // only reachable within rounding of a tangency
        const double sq = nr_range(disc) ? sqrt_nr(disc) : sqrt(disc);
        const double t = k.b + copysign(sq, k.b);  // -s
        double r1, r2;
        if (zero(t)) {
            r1 = 0.0;
            r2 = 0.0;
        } else {
            r1 = nr_range(k.a) ? (-t) * rcp_nr(k.a) : (-t) / k.a;
            r2 = nr_range(t) ? (-k.c) * rcp_nr(t) : (-k.c) / t;
        }
        const bool b_sign = dbits(k.b) < 0;  // sign bit (also for -0.0, as copysign reads it)
        const double lo = b_sign ? r2 : r1, hi = b_sign ? r1 : r2;
        lower = neg(lo) ? 0.0 : lo;                               // max(0, lo)
        upper = (neg(hi) || mag_lt(hi, k.T)) ? hi : k.T;          // min(T, hi)
        if (neg(upper) || mag_lt(upper, lower)) upper = lower;    // (within rounding only)
    }
    *tin = k.t_lo + lower;
    *tout = k.t_lo + upper;
    return true;
}

// Conservative FP32 filter, stage 1: the time extents overlap and the entry MBB meets the query
// MBB expanded by d in every axis. Every bound is rounded outward (entry boxes at build time,
// query boxes at query preparation), so a pair within distance d always passes.
// ea = (xmin - d, ymin - d, zmin - d, w0) rounded down; eb = (xmax + d, ..., w1) rounded up.
static __device__ __forceinline__ bool filter_box(const RecF &r, const float4 &ea, const float4 &eb)
{
    // four independent axis tests, combined as a tree (no short-circuit chain)
    const bool t = (r.t0 < eb.w) & (r.t1 > ea.w);
    const bool x = (r.xmax >= ea.x) & (r.xmin <= eb.x);
    const bool y = (r.ymax >= ea.y) & (r.ymin <= eb.y);
    const bool z = (r.zmax >= ea.z) & (r.zmin <= eb.z);
    return (t & x) & (y & z);
}

// Stage 2: the squared distance between the entry MBB and the query MBB with every subtraction,
// product and sum rounded down (a lower bound of the squared separation over the window),
// against an FP32 upper bound of d^2 that carries 1e-6 relative slack.
// ua = (xmin, ymin, zmin, d2u) rounded down (d2u up); ub = (xmax, ymax, zmax, -) rounded up.
static __device__ __forceinline__ bool filter_gap(const RecF &r, const float4 &ua, const float4 &ub)
{
    float gx = fmaxf(fmaxf(__fsub_rd(r.xmin, ub.x), __fsub_rd(ua.x, r.xmax)), 0.0f);
    float gy = fmaxf(fmaxf(__fsub_rd(r.ymin, ub.y), __fsub_rd(ua.y, r.ymax)), 0.0f);
    float gz = fmaxf(fmaxf(__fsub_rd(r.zmin, ub.z), __fsub_rd(ua.z, r.zmax)), 0.0f);
    float s2 = __fmaf_rd(gz, gz, __fmaf_rd(gy, gy, __fmul_rd(gx, gx)));
    return s2 <= ua.w;
}

// Stage 2 from the d-expanded query box: since eb >= qmax + d and ea <= qmin - d, the gap
// r.min - qmax is at least (r.min - eb) + d, and qmin - r.max at least (ea - r.max) + d; both
// bounds are accumulated rounding down with d_dn <= d, so the result is again a lower bound of
// the squared separation (looser than filter_gap by a few ulps of the coordinates only).
static __device__ __forceinline__ float gap_lo(float a, float b, float d_dn)
{
    return __fadd_rd(__fsub_rd(a, b), d_dn);
}

static __device__ __forceinline__ bool filter_gap_e(const RecF &r, const float4 &ea,
                                                    const float4 &eb, float d_dn, float d2u)
{
    float gx = fmaxf(fmaxf(gap_lo(r.xmin, eb.x, d_dn), gap_lo(ea.x, r.xmax, d_dn)), 0.0f);
    float gy = fmaxf(fmaxf(gap_lo(r.ymin, eb.y, d_dn), gap_lo(ea.y, r.ymax, d_dn)), 0.0f);
    float gz = fmaxf(fmaxf(gap_lo(r.zmin, eb.z, d_dn), gap_lo(ea.z, r.zmax, d_dn)), 0.0f);
    float s2 = __fmaf_rd(gz, gz, __fmaf_rd(gy, gy, __fmul_rd(gx, gx)));
    return s2 <= d2u;
}

}  // namespace ts
