/*
 * ts_oracle.h -- declarations shared by the CPU oracle (ts_oracle.c) and the CPU R-tree baseline
 * (ts_rtree.c). TEST AND BASELINE INFRASTRUCTURE ONLY: the product library never includes this.
 */
#ifndef TS_ORACLE_H
#define TS_ORACLE_H

#include <stdint.h>

/* A segment with its velocity: position p(t) = p0 + v * (t - t0) on [t0, t1] (linear motion
 * between the samples of a trajectory, Sec. 3.1). */
typedef struct {
    double x0, y0, z0, t0, vx, vy, vz, t1;
} orc_seg;

/* Segment i of 8 columns x0, y0, z0, t0, x1, y1, z1, t1, with its velocity. */
void orc_seg_load(const double *const *f, int64_t i, orc_seg *s);

/* The interaction of a query segment and an entry segment (Sec. 3.1): 1 for a hit, with t_in,
 * t_out; s_min = minimum separation over the common window (INFINITY when it is empty). */
int orc_pair(const orc_seg *q, const orc_seg *e, double Ts, double Te, double d,
             double *t_in, double *t_out, double *s_min);

#endif
