/*
 * ts_oracle.c -- CPU oracle for the distance threshold search over historical continuous
 * trajectories (Gowanlock & Casanova, "Towards Efficient Indexing of Spatiotemporal Trajectories
 * on the GPU for Distance Threshold Similarity Searches").
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load this library. The product path (the CUDA library) shares no code, header, table or
 * constant with it, and never calls it.
 *
 * Plain, slow, obviously-correct definitions in FP64 (IEEE round-to-nearest; compiled with
 * -ffp-contract=off so every product and sum is rounded exactly where it is written). Parity pins
 * are in tests/test_oracle_*.py; every function below is pinned by at least one of them.
 *
 * Segment arrays are passed as 8 column pointers in the order x0, y0, z0, t0, x1, y1, z1, t1
 * (start point and end point of a line segment, Sec. 3.1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "ts_oracle.h"

static void seg_load(const double *const *f, int64_t i, orc_seg *s)
{
    double dt = f[7][i] - f[3][i];
    s->x0 = f[0][i];
    s->y0 = f[1][i];
    s->z0 = f[2][i];
    s->t0 = f[3][i];
    s->t1 = f[7][i];
    s->vx = (f[4][i] - f[0][i]) / dt;
    s->vy = (f[5][i] - f[1][i]) / dt;
    s->vz = (f[6][i] - f[2][i]) / dt;
}

void orc_seg_load(const double *const *f, int64_t i, orc_seg *s) { seg_load(f, i, s); }

static double dmax(double a, double b) { return a > b ? a : b; }

/* relative widening of the d-expanded query extents before they are mapped to subbins or cells */
#define EXT_SLACK 1e-12
static double dmin(double a, double b) { return a < b ? a : b; }

/*
 * The interaction between a query segment and an entry segment (the compare() of Alg. 1-3;
 * result tuple (q, l, [t_in, t_out]) of Sec. 3.1). The paper does not write the test out; it is
 * the plain definition: the set of times in the common window at which the two moving points are
 * within distance d.
 *
 * Window: t_lo = max(q.t0, e.t0, Ts), t_hi = min(q.t1, e.t1, Te); pairs need t_lo < t_hi.
 * Relative motion r(tau) = r0 + tau*dv for tau in [0, T], T = t_hi - t_lo, with r0 the relative
 * position at t_lo. |r(tau)|^2 - d^2 = a tau^2 + 2 b tau + c with a = dv.dv, b = r0.dv,
 * c = r0.r0 - d^2. Its non-positive set is one closed interval; roots from the numerically stable
 * pair s/a and c/s with s = -(b + sign(b) sqrt(b^2 - a c)).
 *
 * Returns 1 for a hit and writes t_in, t_out. s_min receives the minimum separation over the
 * window (INFINITY when the window is empty).
 */
int orc_pair(const orc_seg *q, const orc_seg *e, double Ts, double Te, double d,
             double *t_in, double *t_out, double *s_min)
{
    double t_lo = dmax(dmax(q->t0, e->t0), Ts);
    double t_hi = dmin(dmin(q->t1, e->t1), Te);
    if (!(t_lo < t_hi)) {
        *s_min = INFINITY;
        return 0;
    }
    double T = t_hi - t_lo;
    double pqx = q->x0 + q->vx * (t_lo - q->t0);
    double pqy = q->y0 + q->vy * (t_lo - q->t0);
    double pqz = q->z0 + q->vz * (t_lo - q->t0);
    double pex = e->x0 + e->vx * (t_lo - e->t0);
    double pey = e->y0 + e->vy * (t_lo - e->t0);
    double pez = e->z0 + e->vz * (t_lo - e->t0);
    double rx = pqx - pex, ry = pqy - pey, rz = pqz - pez;
    double dvx = q->vx - e->vx, dvy = q->vy - e->vy, dvz = q->vz - e->vz;
    double a = (dvx * dvx + dvy * dvy) + dvz * dvz;
    double b = (rx * dvx + ry * dvy) + rz * dvz;
    double c = ((rx * rx + ry * ry) + rz * rz) - d * d;

    /* minimum separation over the window: at tau* = clamp(-b/a, 0, T) */
    {
        double tau = 0.0;
        if (a > 0.0) {
            tau = -b / a;
            if (tau < 0.0) tau = 0.0;
            if (tau > T) tau = T;
        }
        double sx = rx + tau * dvx, sy = ry + tau * dvy, sz = rz + tau * dvz;
        *s_min = sqrt((sx * sx + sy * sy) + sz * sz);
    }

    double lower, upper;
    if (a == 0.0) {
        if (!(c <= 0.0)) return 0;
        lower = 0.0;
        upper = T;
    } else {
        double disc = b * b - a * c;
        if (disc < 0.0) return 0;
        double sq = sqrt(disc);
        double s = -(b + copysign(sq, b));
        double r1, r2;
        if (s == 0.0) {
            r1 = 0.0;
            r2 = 0.0;
        } else {
            r1 = s / a;
            r2 = c / s;
        }
        lower = dmax(0.0, dmin(r1, r2));
        upper = dmin(T, dmax(r1, r2));
        if (!(lower <= upper)) return 0;
    }
    *t_in = t_lo + lower;
    *t_out = t_lo + upper;
    return 1;
}

/* Evaluate an explicit list of (query, entry) pairs. hit[k] = 1 for a hit; t_in/t_out are written
 * for hits; s_min always. */
void orc_eval_pairs(const double *const *e, const double *const *q, int64_t npairs,
                    const int64_t *qi, const int64_t *ei, double Ts, double Te, double d,
                    int32_t *hit, double *t_in, double *t_out, double *s_min)
{
    for (int64_t k = 0; k < npairs; k++) {
        orc_seg qs, es;
        seg_load(q, qi[k], &qs);
        seg_load(e, ei[k], &es);
        double a = NAN, b = NAN, s = NAN;
        hit[k] = orc_pair(&qs, &es, Ts, Te, d, &a, &b, &s);
        t_in[k] = a;
        t_out[k] = b;
        s_min[k] = s;
    }
}

/* ---------------------------------------------------------------------------------------------
 * All-pairs search (the problem of Sec. 3.1) with exact temporal pruning: entries sorted by
 * t_start (Sec. 4.2 sorts D the same way), and for each query only the entries whose time extent
 * can overlap the clipped window are visited. Pruning removes only pairs whose window is empty,
 * so the result equals the full all-pairs loop (checked by a test).
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    double t0;
    int64_t idx;
} key_t0;

static int cmp_key_t0(const void *pa, const void *pb)
{
    const key_t0 *a = (const key_t0 *)pa, *b = (const key_t0 *)pb;
    if (a->t0 < b->t0) return -1;
    if (a->t0 > b->t0) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

typedef struct {
    int64_t n;
    int64_t *perm;     /* sorted position -> original index */
    double *t0s;       /* t0 in sorted order */
    double *pmax_t1;   /* prefix maximum of t1 in sorted order */
} time_order;

static int time_order_build(int64_t n, const double *t0, const double *t1, time_order *o)
{
    o->n = n;
    o->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    o->t0s = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    o->pmax_t1 = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    key_t0 *k = (key_t0 *)malloc(sizeof(key_t0) * (size_t)(n > 0 ? n : 1));
    if (!o->perm || !o->t0s || !o->pmax_t1 || !k) {
        free(k);
        return -1;
    }
    for (int64_t i = 0; i < n; i++) {
        k[i].t0 = t0[i];
        k[i].idx = i;
    }
    qsort(k, (size_t)n, sizeof(key_t0), cmp_key_t0);
    double run = -INFINITY;
    for (int64_t p = 0; p < n; p++) {
        o->perm[p] = k[p].idx;
        o->t0s[p] = k[p].t0;
        run = dmax(run, t1[k[p].idx]);
        o->pmax_t1[p] = run;
    }
    free(k);
    return 0;
}

static void time_order_free(time_order *o)
{
    free(o->perm);
    free(o->t0s);
    free(o->pmax_t1);
}

/* first sorted position whose prefix-max t1 exceeds w0 (entries before it end at or before w0) */
static int64_t first_pmax_above(const time_order *o, double w0)
{
    int64_t lo = 0, hi = o->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (o->pmax_t1[mid] > w0) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* first sorted position whose t0 is at or after w1 (entries from it on start at or after w1) */
static int64_t first_t0_at_or_above(const time_order *o, double w1)
{
    int64_t lo = 0, hi = o->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (o->t0s[mid] >= w1) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/*
 * Single-threaded search. Writes up to `cap` hits (query index, entry index, t_in, t_out, s_min)
 * in (query, entry time order) order and returns the total number of hits (which may exceed
 * cap). n_tests receives the number of pairs whose window was evaluated. Returns -1 on
 * allocation failure.
 */
int64_t orc_search(int64_t ne, const double *const *e, int64_t nq, const double *const *q,
                   double Ts, double Te, double d, int64_t cap, uint32_t *out_q, uint32_t *out_e,
                   double *out_tin, double *out_tout, double *out_smin, int64_t *n_tests)
{
    time_order o;
    if (time_order_build(ne, e[3], e[7], &o) != 0) return -1;
    int64_t count = 0, tests = 0;
    for (int64_t i = 0; i < nq; i++) {
        orc_seg qs;
        seg_load(q, i, &qs);
        double w0 = dmax(qs.t0, Ts), w1 = dmin(qs.t1, Te);
        if (!(w0 < w1)) continue;
        int64_t lo = first_pmax_above(&o, w0), hi = first_t0_at_or_above(&o, w1);
        for (int64_t p = lo; p < hi; p++) {
            orc_seg es;
            seg_load(e, o.perm[p], &es);
            double tin, tout, smin;
            tests++;
            if (orc_pair(&qs, &es, Ts, Te, d, &tin, &tout, &smin)) {
                if (count < cap) {
                    out_q[count] = (uint32_t)i;
                    out_e[count] = (uint32_t)o.perm[p];
                    out_tin[count] = tin;
                    out_tout[count] = tout;
                    if (out_smin) out_smin[count] = smin;
                }
                count++;
            }
        }
    }
    time_order_free(&o);
    if (n_tests) *n_tests = tests;
    return count;
}

/*
 * The same search over `nthreads` OpenMP threads: a first pass counts every query's hits into
 * cnt[nq] (skipped when have_counts is set: cnt already holds them), and when out_q is not NULL a
 * second pass writes every query's hits at the exclusive prefix sum of the counts, in the same
 * (query, entry time order) order as orc_search. Returns the total hit count (-1 on allocation
 * failure); n_tests receives the pairs evaluated by the counting pass.
 */
int64_t orc_search_mt(int64_t ne, const double *const *e, int64_t nq, const double *const *q,
                      double Ts, double Te, double d, int32_t nthreads, int64_t *cnt,
                      int32_t have_counts, uint32_t *out_q, uint32_t *out_e, double *out_tin,
                      double *out_tout, double *out_smin, int64_t *n_tests)
{
    time_order o;
    if (time_order_build(ne, e[3], e[7], &o) != 0) return -1;
    if (nthreads < 1) nthreads = 1;
    int64_t tests = 0;
    if (!have_counts) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16) reduction(+ : tests)
#endif
        for (int64_t i = 0; i < nq; i++) {
            orc_seg qs;
            seg_load(q, i, &qs);
            cnt[i] = 0;
            double w0 = dmax(qs.t0, Ts), w1 = dmin(qs.t1, Te);
            if (!(w0 < w1)) continue;
            int64_t lo = first_pmax_above(&o, w0), hi = first_t0_at_or_above(&o, w1);
            int64_t c = 0;
            for (int64_t p = lo; p < hi; p++) {
                orc_seg es;
                seg_load(e, o.perm[p], &es);
                double tin, tout, smin;
                tests++;
                c += orc_pair(&qs, &es, Ts, Te, d, &tin, &tout, &smin);
            }
            cnt[i] = c;
        }
        if (n_tests) *n_tests = tests;
    }
    int64_t total = 0;
    for (int64_t i = 0; i < nq; i++) total += cnt[i];
    if (!out_q) {
        time_order_free(&o);
        return total;
    }
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq + 1));
    if (!off) {
        time_order_free(&o);
        return -1;
    }
    off[0] = 0;
    for (int64_t i = 0; i < nq; i++) off[i + 1] = off[i] + cnt[i];
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < nq; i++) {
        if (!cnt[i]) continue;
        orc_seg qs;
        seg_load(q, i, &qs);
        double w0 = dmax(qs.t0, Ts), w1 = dmin(qs.t1, Te);
        int64_t lo = first_pmax_above(&o, w0), hi = first_t0_at_or_above(&o, w1);
        int64_t k = off[i];
        for (int64_t p = lo; p < hi; p++) {
            orc_seg es;
            seg_load(e, o.perm[p], &es);
            double tin, tout, smin;
            if (orc_pair(&qs, &es, Ts, Te, d, &tin, &tout, &smin)) {
                out_q[k] = (uint32_t)i;
                out_e[k] = (uint32_t)o.perm[p];
                out_tin[k] = tin;
                out_tout[k] = tout;
                if (out_smin) out_smin[k] = smin;
                k++;
            }
        }
    }
    free(off);
    time_order_free(&o);
    return total;
}

/*
 * The same search, counting hits only, over `nthreads` OpenMP threads (queries split among
 * threads). Used as the multithreaded CPU baseline. Returns the hit count (-1 on failure);
 * n_tests and n_qsegs (queries with a non-empty clipped window) are written when non-NULL.
 */
int64_t orc_search_count(int64_t ne, const double *const *e, int64_t nq, const double *const *q,
                         double Ts, double Te, double d, int32_t nthreads, int64_t *n_tests,
                         int64_t *n_qsegs)
{
    time_order o;
    if (time_order_build(ne, e[3], e[7], &o) != 0) return -1;
    int64_t count = 0, tests = 0, qsegs = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16) reduction(+ : count, tests, qsegs)
#endif
    for (int64_t i = 0; i < nq; i++) {
        orc_seg qs;
        seg_load(q, i, &qs);
        double w0 = dmax(qs.t0, Ts), w1 = dmin(qs.t1, Te);
        if (!(w0 < w1)) continue;
        qsegs++;
        int64_t lo = first_pmax_above(&o, w0), hi = first_t0_at_or_above(&o, w1);
        for (int64_t p = lo; p < hi; p++) {
            orc_seg es;
            seg_load(e, o.perm[p], &es);
            double tin, tout, smin;
            tests++;
            count += orc_pair(&qs, &es, Ts, Te, d, &tin, &tout, &smin);
        }
    }
    time_order_free(&o);
    if (n_tests) *n_tests = tests;
    if (n_qsegs) *n_qsegs = qsegs;
    return count;
}

int32_t orc_openmp_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------------
 * Temporal index (Sec. 4.2, "Trajectory Indexing"): sort D by t_start (ties by original index),
 * m bins of width b = (t_max - t_min)/m with B_j^start = t_min + j*b, entry l_i in the last bin
 * whose start is <= t_i^start, B_j^end = max(t_min + (j+1)*b, max t_end in B_j), and the index
 * range [B_j^first, B_j^last] of the entries of B_j, stored as offsets off[j] .. off[j+1]-1.
 * ------------------------------------------------------------------------------------------- */
int orc_temporal_index(int64_t n, const double *t0, const double *t1, int32_t m, int64_t *perm,
                       int32_t *bin_of, double *bin_start, double *bin_end, int64_t *bin_off,
                       double *tmin_out, double *b_out)
{
    if (n <= 0 || m <= 0) return -1;
    time_order o;
    if (time_order_build(n, t0, t1, &o) != 0) return -1;
    double tmin = INFINITY, tmax = -INFINITY;
    for (int64_t i = 0; i < n; i++) {
        tmin = dmin(tmin, t0[i]);
        tmax = dmax(tmax, t1[i]);
    }
    double b = (tmax - tmin) / (double)m;
    for (int32_t j = 0; j < m; j++) bin_start[j] = tmin + (double)j * b;
    for (int32_t j = 0; j <= m; j++) bin_off[j] = 0;
    for (int64_t p = 0; p < n; p++) {
        perm[p] = o.perm[p];
        /* last bin whose start is <= t0 */
        int32_t lo = 0, hi = m - 1;
        while (lo < hi) {
            int32_t mid = lo + (hi - lo + 1) / 2;
            if (bin_start[mid] <= o.t0s[p]) lo = mid; else hi = mid - 1;
        }
        bin_of[p] = lo;
        bin_off[lo + 1]++;
    }
    for (int32_t j = 0; j < m; j++) bin_off[j + 1] += bin_off[j];
    for (int32_t j = 0; j < m; j++) {
        double end = tmin + (double)(j + 1) * b;
        for (int64_t p = bin_off[j]; p < bin_off[j + 1]; p++) end = dmax(end, t1[o.perm[p]]);
        bin_end[j] = end;
    }
    *tmin_out = tmin;
    *b_out = b;
    time_order_free(&o);
    return 0;
}

/*
 * Temporal schedule S (Sec. 4.2, "Search Algorithm"): for a query window [w0, w1] the contiguous
 * run of bins from the first bin j_lo whose end (or an earlier bin's end) lies after w0 to the
 * last bin j_hi that starts before w1; E_k = [off[j_lo], off[j_hi+1]) (half-open). Empty when
 * j_lo > j_hi. Bins that end at or before w0, or start at or after w1, cannot hold an entry with a
 * positive-length overlap.
 */
static void temporal_bin_run(int32_t m, const double *bin_start, const double *bin_end, double w0,
                             double w1, int32_t *j_lo, int32_t *j_hi)
{
    int32_t lo = m;
    double run = -INFINITY;
    for (int32_t j = 0; j < m; j++) {
        run = dmax(run, bin_end[j]);
        if (run > w0) {
            lo = j;
            break;
        }
    }
    int32_t hi = -1;
    for (int32_t j = 0; j < m; j++)
        if (bin_start[j] < w1) hi = j;
    *j_lo = lo;
    *j_hi = hi;
}

void orc_temporal_schedule(int32_t m, const double *bin_start, const double *bin_end,
                           const int64_t *bin_off, int64_t nq, const double *w0, const double *w1,
                           int64_t *lo, int64_t *hi)
{
    for (int64_t k = 0; k < nq; k++) {
        int32_t jl, jh;
        temporal_bin_run(m, bin_start, bin_end, w0[k], w1[k], &jl, &jh);
        if (!(w0[k] < w1[k]) || jl > jh) {
            lo[k] = 0;
            hi[k] = 0;
        } else {
            lo[k] = bin_off[jl];
            hi[k] = bin_off[jh + 1];
        }
    }
}

/* ---------------------------------------------------------------------------------------------
 * Uniform 1-D partition used by the spatiotemporal subbins (Sec. 4.3) and the flatly structured
 * grid (Sec. 4.1): v parts with boundaries lo + j*w (j = 0..v-1), the last part unbounded above.
 * Part j is [lo + j*w, lo + (j+1)*w). An extent [a, b] meets part j iff a < lo + (j+1)*w (always
 * true for j = v-1) and b >= lo + j*w.
 * ------------------------------------------------------------------------------------------- */
static int32_t part_of(double x, double lo, double w, int32_t v)
{
    /* largest j in [0, v-1] with lo + j*w <= x, or -1 when x < lo */
    int32_t r = -1;
    for (int32_t j = 0; j < v; j++)
        if (lo + (double)j * w <= x) r = j;
    return r;
}

static int meets_part(double a, double b, double lo, double w, int32_t v, int32_t j)
{
    int below_top = (j == v - 1) ? 1 : (a < lo + (double)(j + 1) * w);
    return below_top && (b >= lo + (double)j * w);
}

/*
 * Subbin geometry of one dimension (Sec. 4.3): extent [min_i min(start,end), max_i max(start,end)]
 * of the entries, v subbins of equal width, with v lowered to floor(extent / max_i |end - start|)
 * when larger so that a subbin is at least as wide as the longest entry (at least 1).
 */
void orc_st_params(int64_t n, const double *emin, const double *emax, int32_t v_req, double *lo,
                   double *w, int32_t *v_eff)
{
    double mn = INFINITY, mx = -INFINITY, longest = 0.0;
    for (int64_t i = 0; i < n; i++) {
        mn = dmin(mn, emin[i]);
        mx = dmax(mx, emax[i]);
        longest = dmax(longest, emax[i] - emin[i]);
    }
    int32_t v = v_req < 1 ? 1 : v_req;
    double ext = mx - mn;
    if (longest > 0.0) {
        double cap = floor(ext / longest);
        if (cap < 1.0) cap = 1.0;
        if ((double)v > cap) v = (int32_t)cap;
    }
    if (!(ext > 0.0)) v = 1;
    *lo = mn;
    *v_eff = v;
    *w = ext / (double)v;
}

/*
 * One dimension's id array of the spatiotemporal index (Sec. 4.3 and Fig. spatiotemporal
 * indexing): ids of the entries (their positions in the time-sorted order) that meet each
 * subbin, subbins B_{i,j} stored in (j, i) lexicographic order, entries of one subbin in time
 * order. off[j*m + i] .. off[j*m + i + 1] - 1 is subbin (i, j)'s range; off has v*m + 1 entries.
 * bin_of[s] is the temporal bin of sorted entry s (non-decreasing in s). Returns the array length
 * (ids written only up to cap).
 */
int64_t orc_st_dim(int64_t n, const double *emin, const double *emax, const int32_t *bin_of,
                   int32_t m, double lo, double w, int32_t v, int64_t cap, uint32_t *ids,
                   int64_t *off)
{
    int64_t len = 0;
    for (int64_t k = 0; k <= (int64_t)v * m; k++) off[k] = 0;
    for (int32_t j = 0; j < v; j++) {
        for (int64_t s = 0; s < n; s++) {
            if (!meets_part(emin[s], emax[s], lo, w, v, j)) continue;
            if (len < cap) ids[len] = (uint32_t)s;
            len++;
            off[(int64_t)j * m + bin_of[s] + 1]++;
        }
    }
    for (int64_t k = 0; k < (int64_t)v * m; k++) off[k + 1] += off[k];
    return len;
}

/*
 * Spatiotemporal schedule (Sec. 4.3, "Search Algorithm"), under the reading that a dimension can
 * serve a query only when the query's MBB expanded by d meets exactly one subbin there (or none:
 * then no entry can be within d and the range is empty). Among such dimensions the one with the
 * fewest ids over the query's temporal bins is picked (lowest dimension on ties); sel = 0, 1, 2
 * for X, Y, Z and [lo, hi) indexes that dimension's id array. Otherwise sel = 3 and [lo, hi) is
 * the temporal range of orc_temporal_schedule.
 * qmin/qmax: 3 pointers each (x, y, z) to the query MBB corners; sub_lo, sub_w, sub_v, off: per
 * dimension.
 */
void orc_st_schedule(int32_t m, const double *bin_start, const double *bin_end,
                     const int64_t *bin_off, const double *sub_lo, const double *sub_w,
                     const int32_t *sub_v, const int64_t *const *off, int64_t nq,
                     const double *const *qmin, const double *const *qmax, const double *w0,
                     const double *w1, double d, int32_t *sel, int64_t *lo, int64_t *hi)
{
    for (int64_t k = 0; k < nq; k++) {
        int32_t jl, jh;
        temporal_bin_run(m, bin_start, bin_end, w0[k], w1[k], &jl, &jh);
        sel[k] = 3;
        if (!(w0[k] < w1[k]) || jl > jh) {
            lo[k] = 0;
            hi[k] = 0;
            continue;
        }
        lo[k] = bin_off[jl];
        hi[k] = bin_off[jh + 1];
        int64_t best = -1;
        for (int dim = 0; dim < 3; dim++) {
            /* d-expanded extent, widened by a relative 1e-12 so that rounding of min - d
             * cannot move the extent past a subbin boundary it truly crosses */
            double a = (qmin[dim][k] - d) - EXT_SLACK * (fabs(qmin[dim][k]) + d);
            double b = (qmax[dim][k] + d) + EXT_SLACK * (fabs(qmax[dim][k]) + d);
            int32_t v = sub_v[dim];
            int32_t pa = part_of(a, sub_lo[dim], sub_w[dim], v);
            int32_t pb = part_of(b, sub_lo[dim], sub_w[dim], v);
            int32_t ja = pa < 0 ? 0 : pa;
            int32_t jb = pb; /* pb <= v-1 by construction; -1 when b is below the first subbin */
            int64_t c_lo, c_hi;
            if (jb < ja) {
                c_lo = 0;
                c_hi = 0;
            } else if (ja == jb) {
                c_lo = off[dim][(int64_t)ja * m + jl];
                c_hi = off[dim][(int64_t)ja * m + jh + 1];
            } else {
                continue;
            }
            if (best < 0 || c_hi - c_lo < best) {
                best = c_hi - c_lo;
                sel[k] = dim;
                lo[k] = c_lo;
                hi[k] = c_hi;
            }
        }
    }
}

/* ---------------------------------------------------------------------------------------------
 * Flatly structured grid (Sec. 4.1): g cells per dimension over the entries' spatial extent,
 * cell h = (cx*g + cy)*g + cz (row-major over (x, y, z)); every entry is listed in each cell its
 * MBB meets (MBB rasterisation); A holds, cell by cell in increasing h, the (time-sorted)
 * positions of the entries of that cell in increasing order; off[h] .. off[h+1]-1 is cell h's
 * range in A (the paper's [A_h^min, A_h^max]; G is the list of h with a non-empty range).
 * lo/w receive the grid origin and cell width per dimension. Returns |A| (written up to cap).
 * emin/emax: 3 pointers each, entries in sorted order.
 * ------------------------------------------------------------------------------------------- */
void orc_grid_params(int64_t n, const double *emin, const double *emax, int32_t g, double *lo,
                     double *w)
{
    double mn = INFINITY, mx = -INFINITY;
    for (int64_t i = 0; i < n; i++) {
        mn = dmin(mn, emin[i]);
        mx = dmax(mx, emax[i]);
    }
    *lo = mn;
    *w = (mx - mn) / (double)g;
}

int64_t orc_fsg(int64_t n, const double *const *emin, const double *const *emax, int32_t g,
                const double *lo, const double *w, int64_t cap, uint32_t *A, int64_t *off)
{
    int64_t ncell = (int64_t)g * g * g;
    int32_t (*rng)[6] = malloc(sizeof(int32_t[6]) * (size_t)(n > 0 ? n : 1));
    if (!rng) return -1;
    for (int64_t s = 0; s < n; s++)
        for (int dim = 0; dim < 3; dim++) {
            int32_t a = part_of(emin[dim][s], lo[dim], w[dim], g);
            int32_t b = part_of(emax[dim][s], lo[dim], w[dim], g);
            rng[s][2 * dim] = a < 0 ? 0 : a;
            rng[s][2 * dim + 1] = b;
        }
    for (int64_t h = 0; h <= ncell; h++) off[h] = 0;
    for (int64_t s = 0; s < n; s++)
        for (int32_t cx = rng[s][0]; cx <= rng[s][1]; cx++)
            for (int32_t cy = rng[s][2]; cy <= rng[s][3]; cy++)
                for (int32_t cz = rng[s][4]; cz <= rng[s][5]; cz++)
                    off[((int64_t)cx * g + cy) * g + cz + 1]++;
    for (int64_t h = 0; h < ncell; h++) off[h + 1] += off[h];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)ncell);
    if (!fill) {
        free(rng);
        return -1;
    }
    memcpy(fill, off, sizeof(int64_t) * (size_t)ncell);
    for (int64_t s = 0; s < n; s++)
        for (int32_t cx = rng[s][0]; cx <= rng[s][1]; cx++)
            for (int32_t cy = rng[s][2]; cy <= rng[s][3]; cy++)
                for (int32_t cz = rng[s][4]; cz <= rng[s][5]; cz++) {
                    int64_t h = ((int64_t)cx * g + cy) * g + cz;
                    int64_t p = fill[h]++;
                    if (p < cap) A[p] = (uint32_t)s;
                }
    free(fill);
    free(rng);
    return off[ncell];
}

/*
 * Candidate generation of the spatial index (Sec. 4.1, "Search Algorithm"): the cells met by the
 * query MBB expanded by d; each such cell's entries are candidates. A pair can appear in several
 * cells; it is kept only from the first cell (lowest cx, cy, cz) the two boxes share, so the
 * candidate list of a query is duplicate-free. Writes, per query, the number of candidates before
 * (n_raw) and after (n_unique) that rule. The entry MBB cell ranges use the same partition as
 * orc_fsg.
 */
void orc_fsg_candidates(int64_t n, const double *const *emin, const double *const *emax,
                        int32_t g, const double *lo, const double *w, const uint32_t *A,
                        const int64_t *off, int64_t nq, const double *const *qmin,
                        const double *const *qmax, double d, int64_t *n_raw, int64_t *n_unique)
{
    for (int64_t k = 0; k < nq; k++) {
        int32_t qa[3], qb[3];
        for (int dim = 0; dim < 3; dim++) {
            int32_t a = part_of(qmin[dim][k] - d, lo[dim], w[dim], g);
            qa[dim] = a < 0 ? 0 : a;
            qb[dim] = part_of(qmax[dim][k] + d, lo[dim], w[dim], g);
        }
        int64_t raw = 0, uniq = 0;
        for (int32_t cx = qa[0]; cx <= qb[0]; cx++)
            for (int32_t cy = qa[1]; cy <= qb[1]; cy++)
                for (int32_t cz = qa[2]; cz <= qb[2]; cz++) {
                    int64_t h = ((int64_t)cx * g + cy) * g + cz;
                    for (int64_t p = off[h]; p < off[h + 1]; p++) {
                        int64_t s = A[p];
                        raw++;
                        int32_t ea[3];
                        for (int dim = 0; dim < 3; dim++) {
                            int32_t a = part_of(emin[dim][s], lo[dim], w[dim], g);
                            ea[dim] = a < 0 ? 0 : a;
                        }
                        int32_t fx = ea[0] > qa[0] ? ea[0] : qa[0];
                        int32_t fy = ea[1] > qa[1] ? ea[1] : qa[1];
                        int32_t fz = ea[2] > qa[2] ? ea[2] : qa[2];
                        if (cx == fx && cy == fy && cz == fz) uniq++;
                    }
                }
        (void)n;
        n_raw[k] = raw;
        n_unique[k] = uniq;
    }
}

/* ---------------------------------------------------------------------------------------------
 * Flatly structured grid with one cell per entry (the Sec. 4.1 grid, each entry listed once in
 * the cell that holds its MBB's minimum corner, so the candidate list of a query is duplicate-free
 * without filtering): A holds, cell by cell in increasing h = (cx*g + cy)*g + cz, the (time-sorted)
 * positions of the entries of that cell in increasing order; off[h] .. off[h+1]-1 is cell h's
 * range. emin: 3 pointers (x, y, z), entries in sorted order. Returns n.
 * ------------------------------------------------------------------------------------------- */
int64_t orc_grid1(int64_t n, const double *const *emin, int32_t g, const double *lo,
                  const double *w, uint32_t *A, int64_t *off)
{
    int64_t ncell = (int64_t)g * g * g;
    int64_t *cell = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cell) return -1;
    for (int64_t h = 0; h <= ncell; h++) off[h] = 0;
    for (int64_t s = 0; s < n; s++) {
        int32_t c[3];
        for (int dim = 0; dim < 3; dim++) {
            int32_t a = part_of(emin[dim][s], lo[dim], w[dim], g);
            c[dim] = a < 0 ? 0 : a;
        }
        cell[s] = ((int64_t)c[0] * g + c[1]) * g + c[2];
        off[cell[s] + 1]++;
    }
    for (int64_t h = 0; h < ncell; h++) off[h + 1] += off[h];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)ncell);
    if (!fill) {
        free(cell);
        return -1;
    }
    memcpy(fill, off, sizeof(int64_t) * (size_t)ncell);
    for (int64_t s = 0; s < n; s++) A[fill[cell[s]]++] = (uint32_t)s;
    free(fill);
    free(cell);
    return n;
}

/*
 * Candidates of a query in the one-cell-per-entry grid: an entry within d of the query has its
 * MBB minimum corner in [qmin - d - longest, qmax + d] per axis (longest = the largest extent of
 * an entry along that axis), widened by a relative 1e-12 against rounding. The cells meeting that
 * box are read as z-runs, one per (cx, cy). Per query (window [w0, w1] must have positive length,
 * else 0): the number of runs and of candidates (the runs' total length).
 */
void orc_grid1_candidates(int32_t g, const double *lo, const double *w, const double *longest,
                          const int64_t *off, int64_t nq, const double *const *qmin,
                          const double *const *qmax, const double *w0, const double *w1, double d,
                          int64_t *n_runs, int64_t *n_cand)
{
    for (int64_t k = 0; k < nq; k++) {
        n_runs[k] = 0;
        n_cand[k] = 0;
        if (!(w0[k] < w1[k])) continue;
        int32_t ca[3], cb[3];
        int empty = 0;
        for (int dim = 0; dim < 3; dim++) {
            double a = ((qmin[dim][k] - d) - longest[dim]) -
                       EXT_SLACK * ((fabs(qmin[dim][k]) + d) + longest[dim]);
            double b = (qmax[dim][k] + d) + EXT_SLACK * (fabs(qmax[dim][k]) + d);
            int32_t pa = part_of(a, lo[dim], w[dim], g);
            int32_t pb = part_of(b, lo[dim], w[dim], g);
            ca[dim] = pa < 0 ? 0 : pa;
            cb[dim] = pb;
            if (pb < ca[dim]) empty = 1;
        }
        if (empty) continue;
        n_runs[k] = (int64_t)(cb[0] - ca[0] + 1) * (cb[1] - ca[1] + 1);
        for (int32_t cx = ca[0]; cx <= cb[0]; cx++)
            for (int32_t cy = ca[1]; cy <= cb[1]; cy++) {
                int64_t row = ((int64_t)cx * g + cy) * g;
                n_cand[k] += off[row + cb[2] + 1] - off[row + ca[2]];
            }
    }
}
