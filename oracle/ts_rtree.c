/*
 * ts_rtree.c -- CPU in-memory R-tree baseline for the distance threshold search (the CPU
 * comparator of the paper's experiments, Sec. 5: trajectories cut into groups of r consecutive
 * segments, one 4-D minimum bounding box (x, y, z, t) per group, the boxes indexed by an R-tree,
 * queries run in parallel with OpenMP).
 *
 * BENCHMARK AND TEST INFRASTRUCTURE ONLY: the benchmark's CPU-baseline leg and the tests load it
 * (it lives beside the oracle, in the same library); the product library never does.
 *
 * Build: the group boxes are bulk-loaded with Sort-Tile-Recursive packing (Leutenegger, Lopez
 * and Edgington, "STR: a simple and efficient algorithm for R-tree packing", ICDE 1997),
 * generalised to four dimensions: sort the boxes by the centre of one dimension, cut them into
 * equal slabs, sort every slab by the next dimension, and so on, then pack runs of RT_FAN boxes
 * into nodes; every level above packs runs of RT_FAN nodes of the level below, in that order.
 *
 * Search: for every query segment, the boxes that meet its window [max(t0, Ts), min(t1, Te)] and
 * its MBB widened by d in x, y and z (closed intervals; rounding of min - d and max + d is
 * monotone, so a segment within d of the query always meets the widened box); the r segments of
 * every such leaf group go through the oracle's interaction test (orc_pair), so the match set is
 * the oracle's. A segment belongs to one group, so no pair is reported twice.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "ts_oracle.h"

#define RT_FAN 16  /* children per node */

typedef struct {
    double lo[4], hi[4];  /* x, y, z, t */
} rt_box;

typedef struct {
    int64_t n_seg;           /* database segments */
    const double *cols[8];   /* the caller's columns (kept by the caller while the tree lives) */
    int64_t n_groups;        /* leaf boxes: groups of up to r consecutive segments */
    int64_t *g_first;        /* first segment of every group (n_groups + 1, in leaf order) */
    int64_t *g_seg;          /* segments in group order */
    int n_levels;            /* level 0 = the group boxes, the last level = the root */
    int64_t *lv_n;           /* boxes per level */
    rt_box **lv_box;         /* boxes per level, in packed order */
    int64_t **lv_child;      /* per level > 0: first child of every node (n + 1) */
} rt_tree;

static double dmin2(double a, double b) { return a < b ? a : b; }
static double dmax2(double a, double b) { return a > b ? a : b; }

/* ---------------------------------------------------------------------------------------------
 * STR packing
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    double key;  /* twice the box centre in the sorted dimension */
    int64_t idx;
} key_idx;

static int cmp_key(const void *a, const void *b)
{
    const key_idx *x = (const key_idx *)a, *y = (const key_idx *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);  /* a total order: ties by index */
}

/* Order the boxes idx[0..n) for packing: sort by the centre of dimension dims[k], cut into slabs
 * of whole nodes, recurse on the next dimension inside every slab (slabs in parallel). */
static void str_order(const rt_box *box, int64_t *idx, int64_t n, const int *dims, int k, int nd,
                      key_idx *tmp)
{
    if (n <= RT_FAN || k >= nd) return;
    const int d = dims[k];
    for (int64_t i = 0; i < n; i++) {
        tmp[i].key = box[idx[i]].lo[d] + box[idx[i]].hi[d];
        tmp[i].idx = idx[i];
    }
    qsort(tmp, (size_t)n, sizeof(key_idx), cmp_key);
    for (int64_t i = 0; i < n; i++) idx[i] = tmp[i].idx;
    if (k + 1 >= nd) return;
    const double nodes = ceil((double)n / RT_FAN);
    /* slabs per remaining dimension: nodes^(1 / dimensions left) */
    const int64_t slabs = (int64_t)ceil(pow(nodes, 1.0 / (double)(nd - k)));
    const int64_t per = (int64_t)ceil(nodes / (double)slabs) * RT_FAN;  /* boxes per slab */
    const int64_t ns = (n + per - 1) / per;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) if (k == 0)
#endif
    for (int64_t j = 0; j < ns; j++) {
        const int64_t s0 = j * per;
        str_order(box, idx + s0, (s0 + per < n ? per : n - s0), dims, k + 1, nd, tmp + s0);
    }
}

static void box_union(rt_box *u, const rt_box *b)
{
    for (int d = 0; d < 4; d++) {
        u->lo[d] = dmin2(u->lo[d], b->lo[d]);
        u->hi[d] = dmax2(u->hi[d], b->hi[d]);
    }
}

static void box_empty(rt_box *u)
{
    for (int d = 0; d < 4; d++) {
        u->lo[d] = INFINITY;
        u->hi[d] = -INFINITY;
    }
}

void orc_rtree_free(void *h);

/* Build the tree over n segments (8 columns), r consecutive segments of a trajectory per leaf
 * box; consecutive input segments belong to one trajectory when the first ends where and when
 * the second starts. Returns NULL on allocation failure. */
void *orc_rtree_build(int64_t n, const double *const *e, int32_t r)
{
    if (r < 1) r = 1;
    rt_tree *t = (rt_tree *)calloc(1, sizeof(rt_tree));
    if (!t) return NULL;
    t->n_seg = n;
    for (int c = 0; c < 8; c++) t->cols[c] = e[c];
    /* groups of up to r consecutive segments within a trajectory */
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!first) {
        free(t);
        return NULL;
    }
    int64_t ng = 0;
    for (int64_t i = 0; i < n;) {
        first[ng++] = i;
        int64_t j = i + 1;
        while (j < n && j - i < r && e[7][j - 1] == e[3][j] && e[4][j - 1] == e[0][j] &&
               e[5][j - 1] == e[1][j] && e[6][j - 1] == e[2][j])
            j++;
        i = j;
    }
    first[ng] = n;
    rt_box *gb = (rt_box *)malloc(sizeof(rt_box) * (size_t)(ng ? ng : 1));
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng ? ng : 1));
    if (!gb || !ord) {
        free(first);
        free(gb);
        free(ord);
        free(t);
        return NULL;
    }
    for (int64_t g = 0; g < ng; g++) {
        box_empty(&gb[g]);
        for (int64_t i = first[g]; i < first[g + 1]; i++) {
            rt_box s;
            s.lo[0] = dmin2(e[0][i], e[4][i]);
            s.hi[0] = dmax2(e[0][i], e[4][i]);
            s.lo[1] = dmin2(e[1][i], e[5][i]);
            s.hi[1] = dmax2(e[1][i], e[5][i]);
            s.lo[2] = dmin2(e[2][i], e[6][i]);
            s.hi[2] = dmax2(e[2][i], e[6][i]);
            s.lo[3] = e[3][i];
            s.hi[3] = e[7][i];
            box_union(&gb[g], &s);
        }
    }
    /* level 0: the group boxes in STR order (time first: trajectories are long-lived) */
    const int dims[4] = {3, 0, 1, 2};
    for (int64_t g = 0; g < ng; g++) ord[g] = g;
    key_idx *tmp = (key_idx *)malloc(sizeof(key_idx) * (size_t)(ng ? ng : 1));
    if (!tmp) {
        free(first);
        free(gb);
        free(ord);
        free(t);
        return NULL;
    }
    str_order(gb, ord, ng, dims, 0, 4, tmp);
    free(tmp);
    t->n_groups = ng;
    t->g_first = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng + 1));
    t->g_seg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int max_levels = 64;
    t->lv_n = (int64_t *)calloc((size_t)max_levels, sizeof(int64_t));
    t->lv_box = (rt_box **)calloc((size_t)max_levels, sizeof(rt_box *));
    t->lv_child = (int64_t **)calloc((size_t)max_levels, sizeof(int64_t *));
    t->lv_box[0] = (rt_box *)malloc(sizeof(rt_box) * (size_t)(ng ? ng : 1));
    int64_t k = 0;
    for (int64_t p = 0; p < ng; p++) {
        const int64_t g = ord[p];
        t->g_first[p] = k;
        for (int64_t i = first[g]; i < first[g + 1]; i++) t->g_seg[k++] = i;
        t->lv_box[0][p] = gb[g];
    }
    t->g_first[ng] = k;
    t->lv_n[0] = ng;
    free(first);
    free(gb);
    free(ord);
    /* upper levels: runs of RT_FAN boxes of the level below (already in packing order) */
    int lv = 0;
    while (t->lv_n[lv] > 1 && lv + 1 < max_levels) {
        const int64_t nb = t->lv_n[lv];
        const int64_t nn = (nb + RT_FAN - 1) / RT_FAN;
        rt_box *up = (rt_box *)malloc(sizeof(rt_box) * (size_t)nn);
        int64_t *ch = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
        for (int64_t u = 0; u < nn; u++) {
            ch[u] = u * RT_FAN;
            box_empty(&up[u]);
            const int64_t end = (u + 1) * RT_FAN < nb ? (u + 1) * RT_FAN : nb;
            for (int64_t c = u * RT_FAN; c < end; c++) box_union(&up[u], &t->lv_box[lv][c]);
        }
        ch[nn] = nb;
        lv++;
        t->lv_box[lv] = up;
        t->lv_child[lv] = ch;
        t->lv_n[lv] = nn;
    }
    t->n_levels = lv + 1;
    if (!t->g_first || !t->g_seg || !t->lv_box[0]) {
        orc_rtree_free(t);
        return NULL;
    }
    return t;
}

void orc_rtree_free(void *h)
{
    rt_tree *t = (rt_tree *)h;
    if (!t) return;
    for (int l = 0; l < 64 && t->lv_box; l++) {
        free(t->lv_box[l]);
        if (t->lv_child) free(t->lv_child[l]);
    }
    free(t->lv_box);
    free(t->lv_child);
    free(t->lv_n);
    free(t->g_first);
    free(t->g_seg);
    free(t);
}

/* Leaf boxes and levels of a tree (for tests): n_groups, n_levels. */
void orc_rtree_shape(const void *h, int64_t *n_groups, int32_t *n_levels)
{
    const rt_tree *t = (const rt_tree *)h;
    *n_groups = t->n_groups;
    *n_levels = t->n_levels;
}

/* ---------------------------------------------------------------------------------------------
 * search
 * ------------------------------------------------------------------------------------------- */
static int meets(const rt_box *b, const double *lo, const double *hi)
{
    for (int d = 0; d < 4; d++)
        if (b->hi[d] < lo[d] || b->lo[d] > hi[d]) return 0;
    return 1;
}

/* One query segment: visits the leaf groups whose boxes meet its widened box and tests their
 * segments. emit (optional) receives up to cap hits (entry index, t_in, t_out). Returns the hit
 * count; *tests counts the interaction tests made. */
static int64_t query_one(const rt_tree *t, const double *const *qc, int64_t i, double Ts,
                         double Te, double d, int64_t *tests, int64_t *e_out, double *tin_out,
                         double *tout_out, int64_t cap)
{
    orc_seg qs;
    orc_seg_load(qc, i, &qs);
    const orc_seg *q = &qs;
    const double w0 = dmax2(q->t0, Ts), w1 = dmin2(q->t1, Te);
    if (!(w0 < w1) || t->n_groups == 0) return 0;
    /* the query's MBB from its end points, widened by d */
    double lo[4], hi[4];
    for (int k = 0; k < 3; k++) {
        lo[k] = dmin2(qc[k][i], qc[k + 4][i]) - d;
        hi[k] = dmax2(qc[k][i], qc[k + 4][i]) + d;
    }
    lo[3] = w0;
    hi[3] = w1;
    /* depth-first over the levels with an explicit stack of (level, node) */
    int64_t stack_node[64 * RT_FAN];
    int stack_lv[64 * RT_FAN];
    int sp = 0;
    const int top = t->n_levels - 1;
    stack_node[sp] = 0;
    stack_lv[sp] = top;
    sp++;
    int64_t hits = 0;
    while (sp > 0) {
        sp--;
        const int l = stack_lv[sp];
        const int64_t nd = stack_node[sp];
        if (!meets(&t->lv_box[l][nd], lo, hi)) continue;
        if (l == 0) {
            for (int64_t k = t->g_first[nd]; k < t->g_first[nd + 1]; k++) {
                orc_seg es;
                orc_seg_load(t->cols, t->g_seg[k], &es);
                double tin, tout, smin;
                (*tests)++;
                if (orc_pair(q, &es, Ts, Te, d, &tin, &tout, &smin)) {
                    if (e_out && hits < cap) {
                        e_out[hits] = t->g_seg[k];
                        tin_out[hits] = tin;
                        tout_out[hits] = tout;
                    }
                    hits++;
                }
            }
            continue;
        }
        const int64_t *ch = t->lv_child[l];
        for (int64_t c = ch[nd + 1]; c-- > ch[nd];) {
            stack_node[sp] = c;
            stack_lv[sp] = l - 1;
            sp++;
        }
    }
    return hits;
}

/* Hit count of the search on nthreads OpenMP threads; *n_tests = interaction tests made,
 * *n_qsegs = query segments with a positive overlap with [Ts, Te]. */
int64_t orc_rtree_count(const void *h, int64_t nq, const double *const *q, double Ts, double Te,
                        double d, int32_t nthreads, int64_t *n_tests, int64_t *n_qsegs)
{
    const rt_tree *t = (const rt_tree *)h;
    int64_t count = 0, tests = 0, qsegs = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16) reduction(+ : count, tests, qsegs)
#endif
    for (int64_t i = 0; i < nq; i++) {
        if (!(dmax2(q[3][i], Ts) < dmin2(q[7][i], Te))) continue;
        qsegs++;
        int64_t nt = 0;
        count += query_one(t, q, i, Ts, Te, d, &nt, NULL, NULL, NULL, 0);
        tests += nt;
    }
    if (n_tests) *n_tests = tests;
    if (n_qsegs) *n_qsegs = qsegs;
    return count;
}

/* Every hit of the search (query index, entry index, t_in, t_out), query by query, into arrays
 * of cap rows; returns the hit count (rows are written only when it is at most cap). */
int64_t orc_rtree_search(const void *h, int64_t nq, const double *const *q, double Ts, double Te,
                         double d, int32_t nthreads, int64_t cap, int64_t *q_out, int64_t *e_out,
                         double *tin_out, double *tout_out)
{
    const rt_tree *t = (const rt_tree *)h;
    int64_t *cnt = (int64_t *)calloc((size_t)(nq + 1), sizeof(int64_t));
    if (!cnt) return -1;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < nq; i++) {
        int64_t nt = 0;
        cnt[i + 1] = query_one(t, q, i, Ts, Te, d, &nt, NULL, NULL, NULL, 0);
    }
    for (int64_t i = 0; i < nq; i++) cnt[i + 1] += cnt[i];
    const int64_t total = cnt[nq];
    if (total <= cap) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < nq; i++) {
            int64_t nt = 0;
            const int64_t o = cnt[i];
            const int64_t k = query_one(t, q, i, Ts, Te, d, &nt, e_out + o, tin_out + o,
                                        tout_out + o, cnt[i + 1] - o);
            for (int64_t j = 0; j < k; j++) q_out[o + j] = i;
        }
    }
    free(cnt);
    return total;
}
