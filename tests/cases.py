"""Hand-built segment sets with closed-form answers, and small random cases.

Every expected value here is derived by hand from the geometry of the case (written next to
it), never by evaluating the search formula.
"""
from __future__ import annotations

import numpy as np

from paper_1410_2698_gb300.workloads import Segments


def seg(p0, t0, p1, t1):
    """One segment as a row x0, y0, z0, t0, x1, y1, z1, t1."""
    return [float(p0[0]), float(p0[1]), float(p0[2]), float(t0),
            float(p1[0]), float(p1[1]), float(p1[2]), float(t1)]


def segset(rows):
    return Segments.from_matrix(np.array(rows, dtype=np.float64).reshape(-1, 8))


def random_segments(rng, n, box=10.0, t_range=(0.0, 10.0), max_len=3.0, max_dur=3.0,
                    stationary_frac=0.0):
    """n random segments with overlapping time extents (for sampling checks)."""
    p0 = rng.uniform(0.0, box, size=(n, 3))
    p1 = p0 + rng.uniform(-max_len, max_len, size=(n, 3))
    if stationary_frac > 0:
        still = rng.uniform(size=n) < stationary_frac
        p1[still] = p0[still]
    t0 = rng.uniform(t_range[0], t_range[1], size=n)
    t1 = t0 + rng.uniform(0.05, max_dur, size=n)
    m = np.concatenate([p0, t0[:, None], p1, t1[:, None]], axis=1)
    return Segments.from_matrix(m)


def sample_separation(q: Segments, e: Segments, qi, ei, t):
    """|p_q(t) - p_e(t)| by linear interpolation between the endpoints (p0 + (p1-p0) * frac),
    a different formulation from the velocity form used by the search."""
    def pos(s: Segments, i, tt):
        f = (tt - s.t0[i]) / (s.t1[i] - s.t0[i])
        return np.stack([s.x0[i] + (s.x1[i] - s.x0[i]) * f,
                         s.y0[i] + (s.y1[i] - s.y0[i]) * f,
                         s.z0[i] + (s.z1[i] - s.z0[i]) * f], axis=-1)
    return np.linalg.norm(pos(q, qi, t) - pos(e, ei, t), axis=-1)
