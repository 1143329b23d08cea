"""Seeded synthetic trajectory workloads.

This module only draws random trajectories and cuts them into line segments. It holds none of
the search arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The shapes follow the datasets of the paper's experimental evaluation (Sec. 5.1): uniform random
walks (Random-1M), a dense random-walk cube (Random-dense) and a two-galaxy merger (Merger). The
merger data itself is not available, so a two-Plummer-sphere stand-in is drawn instead. Every
recipe is written out in the function that draws it. Trajectories are polylines of 4-D samples
(x, y, z, t); segment k of a trajectory joins samples k and k+1 (Sec. 3.1).

Seeds: workload ``i`` uses ``numpy.random.PCG64(1410 + i)`` for the database and a separate
``PCG64(1410 + i + 1000)`` stream for choosing the query trajectories.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1410


@dataclasses.dataclass
class Segments:
    """Structure-of-arrays FP64 line segments (Sec. 3.1): start point, end point, trajectory id."""

    x0: np.ndarray
    y0: np.ndarray
    z0: np.ndarray
    t0: np.ndarray
    x1: np.ndarray
    y1: np.ndarray
    z1: np.ndarray
    t1: np.ndarray
    traj: np.ndarray  # uint32 trajectory id of every segment

    FIELDS = ("x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1")

    @property
    def n(self) -> int:
        return int(self.x0.shape[0])

    def arrays(self):
        return [getattr(self, f) for f in self.FIELDS]

    def take(self, idx) -> "Segments":
        idx = np.asarray(idx)
        return Segments(*[np.ascontiguousarray(getattr(self, f)[idx]) for f in self.FIELDS],
                        traj=np.ascontiguousarray(self.traj[idx]))

    def as_matrix(self) -> np.ndarray:
        """(n, 8) matrix in the field order x0, y0, z0, t0, x1, y1, z1, t1."""
        return np.stack(self.arrays(), axis=1)

    @staticmethod
    def from_matrix(m: np.ndarray, traj=None) -> "Segments":
        m = np.asarray(m, dtype=np.float64)
        if m.ndim != 2 or m.shape[1] != 8:
            raise ValueError("expected an (n, 8) matrix")
        cols = [np.ascontiguousarray(m[:, i]) for i in range(8)]
        if traj is None:
            traj = np.zeros(m.shape[0], dtype=np.uint32)
        return Segments(*cols, traj=np.ascontiguousarray(traj, dtype=np.uint32))


@dataclasses.dataclass
class Workload:
    name: str
    db: Segments
    queries: Segments
    t_start: float
    t_end: float
    distances: tuple
    db_traj_first: np.ndarray  # first segment index of every database trajectory
    query_traj_ids: np.ndarray  # database trajectory ids the queries were drawn from


def samples_to_segments(pos: np.ndarray, t: np.ndarray, traj_ids=None) -> Segments:
    """Cut trajectories of samples into segments.

    pos: (n_traj, n_samples, 3) positions, t: (n_traj, n_samples) times. Segment k of trajectory j
    joins samples k and k+1, and segments of one trajectory are stored contiguously in temporal
    order (Sec. 3.1).
    """
    pos = np.asarray(pos, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n_traj, n_s, _ = pos.shape
    if n_s < 2:
        raise ValueError("a trajectory needs at least two samples")
    a = pos[:, :-1, :].reshape(-1, 3)
    b = pos[:, 1:, :].reshape(-1, 3)
    ta = t[:, :-1].reshape(-1)
    tb = t[:, 1:].reshape(-1)
    if traj_ids is None:
        traj_ids = np.arange(n_traj, dtype=np.uint32)
    tid = np.repeat(np.asarray(traj_ids, dtype=np.uint32), n_s - 1)
    c = np.ascontiguousarray
    return Segments(c(a[:, 0]), c(a[:, 1]), c(a[:, 2]), c(ta), c(b[:, 0]), c(b[:, 1]), c(b[:, 2]),
                    c(tb), traj=tid)


def _random_walk(rng, n_traj, n_samples, box, t0_range, sigma, reflect=None):
    """Gaussian random walks with dt = 1 and N(0, sigma^2) steps per axis."""
    p0 = rng.uniform(box[0], box[1], size=(n_traj, 1, 3))
    steps = rng.normal(0.0, sigma, size=(n_traj, n_samples - 1, 3))
    pos = np.concatenate([p0, p0 + np.cumsum(steps, axis=1)], axis=1)
    if reflect is not None:
        lo, hi = reflect
        width = hi - lo
        # Reflecting walls: fold the free walk back into [lo, hi] (x<lo -> 2lo-x, x>hi -> 2hi-x,
        # repeated, i.e. a triangle wave of period 2*width).
        u = np.mod(pos - lo, 2.0 * width)
        pos = lo + np.where(u > width, 2.0 * width - u, u)
    if t0_range[0] == t0_range[1]:
        t_start = np.full((n_traj, 1), float(t0_range[0]))
    else:
        t_start = rng.uniform(t0_range[0], t0_range[1], size=(n_traj, 1))
    t = t_start + np.arange(n_samples, dtype=np.float64)[None, :]
    return pos, t


def _query_from_traj(db: Segments, n_seg_per_traj: int, traj_ids) -> Segments:
    idx = (np.asarray(traj_ids, dtype=np.int64)[:, None] * n_seg_per_traj
           + np.arange(n_seg_per_traj, dtype=np.int64)[None, :]).reshape(-1)
    return db.take(idx)


def tiny(seed_offset: int = 0) -> Workload:
    """Tiny plain search: 1,000 trajectories x 21 samples (20,000 segments) starting uniform in
    [0,100]^3 at t0 uniform in [0,50], dt = 1, per-step displacement N(0,1) per axis; 100 query
    trajectories drawn without replacement from the database; query interval [0,70]; d = 5."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 0 + seed_offset))
    qrng = np.random.Generator(np.random.PCG64(SEED_BASE + 0 + 1000 + seed_offset))
    n_traj, n_s = 1000, 21
    pos, t = _random_walk(rng, n_traj, n_s, (0.0, 100.0), (0.0, 50.0), 1.0)
    db = samples_to_segments(pos, t)
    q_traj = np.sort(qrng.choice(n_traj, size=100, replace=False))
    q = _query_from_traj(db, n_s - 1, q_traj)
    return Workload("tiny-20k", db, q, 0.0, 70.0, (5.0,),
                    np.arange(n_traj) * (n_s - 1), q_traj)


def random_walk_1m(seed_offset: int = 0, n_traj: int = 2500, n_samples: int = 401) -> Workload:
    """Random-walk 1M (stand-in for the paper's Random-1M, Sec. 5.1): 2,500 trajectories x 401
    samples (1,000,000 segments) starting uniform in [0,1000]^3, t0 uniform in [0,100], dt = 1,
    steps N(0,2^2) per axis; queries = 1% of the trajectories; full time span; d in {1,5,10,25}."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1 + seed_offset))
    qrng = np.random.Generator(np.random.PCG64(SEED_BASE + 1 + 1000 + seed_offset))
    pos, t = _random_walk(rng, n_traj, n_samples, (0.0, 1000.0), (0.0, 100.0), 2.0)
    db = samples_to_segments(pos, t)
    n_q = max(1, n_traj // 100)
    q_traj = np.sort(qrng.choice(n_traj, size=n_q, replace=False))
    q = _query_from_traj(db, n_samples - 1, q_traj)
    return Workload("random-walk-1m", db, q, float(t.min()), float(t.max()),
                    (1.0, 5.0, 10.0, 25.0), np.arange(n_traj) * (n_samples - 1), q_traj)


def dense(seed_offset: int = 0, n_traj: int = 20000, n_samples: int = 101,
          n_query_traj: int = 500) -> Workload:
    """Dense random (stand-in for Random-dense, Sec. 5.1): 20,000 trajectories x 101 samples
    (2,000,000 segments) in [0,50]^3 with reflecting walls, all starting at t = 0, dt = 1, steps
    N(0,0.5^2) per axis; 500 query trajectories; d in {0.5, 2}."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 2 + seed_offset))
    qrng = np.random.Generator(np.random.PCG64(SEED_BASE + 2 + 1000 + seed_offset))
    pos, t = _random_walk(rng, n_traj, n_samples, (0.0, 50.0), (0.0, 0.0), 0.5,
                          reflect=(0.0, 50.0))
    db = samples_to_segments(pos, t)
    q_traj = np.sort(qrng.choice(n_traj, size=min(n_query_traj, n_traj), replace=False))
    q = _query_from_traj(db, n_samples - 1, q_traj)
    return Workload("dense-2m", db, q, 0.0, float(n_samples - 1), (0.5, 2.0),
                    np.arange(n_traj) * (n_samples - 1), q_traj)


def _plummer_radii(rng, n, a, r_max):
    """Plummer-sphere radii by inverse CDF, r = a / sqrt(X^(-2/3) - 1), X ~ U(0,1), with radii
    above r_max redrawn (rejection)."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        x = rng.uniform(0.0, 1.0, size=n - filled)
        x = x[x > 0.0]
        r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        r = r[np.isfinite(r) & (r <= r_max)]
        out[filled:filled + r.size] = r
        filled += r.size
    return out


def _isotropic(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def merger_like(seed_offset: int = 0, n_per_cluster: int = 50000, n_samples: int = 201,
                n_query_traj: int = 2000, query_seed_offset=None) -> Workload:
    """Merger-like (stand-in for the Merger dataset, Sec. 5.1, which is not available): two
    Plummer spheres of 50,000 particles each (scale radius a = 10, radii truncated at 10a by
    rejection, isotropic directions), centred at (-100,-5,0) and (+100,+5,0) and moving at
    +(0.5,0,0) and -(0.5,0,0) (approaching at relative speed 1 on lines offset by 10 in y). Each
    particle follows x_{k+1} = x_k + v_bulk*dt + N(0, 0.1^2) per axis; 201 samples at dt = 1 on
    t in [0,200] (20,000,000 segments). Queries: 2,000 trajectories, 1,000 per cluster, drawn
    among the particles whose initial radius is below a (another draw of them with
    query_seed_offset, the same database). d in {1, 5}."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 3 + seed_offset))
    qoff = seed_offset if query_seed_offset is None else query_seed_offset
    qrng = np.random.Generator(np.random.PCG64(SEED_BASE + 3 + 1000 + qoff))
    a = 10.0
    centres = np.array([[-100.0, -5.0, 0.0], [100.0, 5.0, 0.0]])
    vbulk = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    n = 2 * n_per_cluster
    pos = np.empty((n, n_samples, 3))
    r_all = np.empty(n)
    for c in range(2):
        sl = slice(c * n_per_cluster, (c + 1) * n_per_cluster)
        r = _plummer_radii(rng, n_per_cluster, a, 10.0 * a)
        r_all[sl] = r
        p0 = centres[c] + r[:, None] * _isotropic(rng, n_per_cluster)
        steps = vbulk[c][None, None, :] + rng.normal(0.0, 0.1, size=(n_per_cluster, n_samples - 1, 3))
        pos[sl, 0, :] = p0
        pos[sl, 1:, :] = p0[:, None, :] + np.cumsum(steps, axis=1)
    t = np.broadcast_to(np.arange(n_samples, dtype=np.float64)[None, :], (n, n_samples))
    db = samples_to_segments(pos, t)
    q_ids = []
    per = n_query_traj // 2
    for c in range(2):
        base = c * n_per_cluster
        core = np.nonzero(r_all[base:base + n_per_cluster] < a)[0] + base
        q_ids.append(qrng.choice(core, size=min(per, core.size), replace=False))
    q_traj = np.sort(np.concatenate(q_ids))
    q = _query_from_traj(db, n_samples - 1, q_traj)
    nseg = n * (n_samples - 1)
    return Workload(f"merger-like-{nseg // 1000000}m", db, q, 0.0, float(n_samples - 1),
                    (1.0, 5.0), np.arange(n) * (n_samples - 1), q_traj)


@dataclasses.dataclass
class Request:
    queries: Segments
    t_start: float
    t_end: float
    d: float
    arrival_s: float


def served_stream(db_workload: Workload, n_requests: int = 10000, rate_per_s: float = 100.0,
                  seed_offset: int = 0, max_traj: int = 5000, len_range=(10, 200)):
    """Served query stream on a resident database: Poisson arrivals at ``rate_per_s``; each
    request holds n_traj ~ log-uniform[1, max_traj] query trajectories, each a random database
    trajectory restricted to a contiguous run of L ~ U{len_range} segments; the request's
    interval is the span of its runs and d ~ log-uniform[0.5, 10]."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4 + seed_offset))
    db = db_workload.db
    first = np.asarray(db_workload.db_traj_first, dtype=np.int64)
    n_traj = first.size
    seg_per = np.diff(np.append(first, db.n))
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        k = int(round(math.exp(rng.uniform(0.0, math.log(max_traj)))))
        k = max(1, min(k, max_traj))
        trajs = rng.integers(0, n_traj, size=k)
        lens = rng.integers(len_range[0], len_range[1] + 1, size=k)
        lens = np.minimum(lens, seg_per[trajs])
        starts = rng.integers(0, seg_per[trajs] - lens + 1)
        idx = np.concatenate([first[tr] + s + np.arange(L) for tr, s, L in zip(trajs, starts, lens)])
        q = db.take(idx)
        d = float(math.exp(rng.uniform(math.log(0.5), math.log(10.0))))
        out.append(Request(q, float(q.t0.min()), float(q.t1.max()), d, t))
    return out


WORKLOADS = {
    "tiny": tiny,
    "random-walk-1m": random_walk_1m,
    "dense": dense,
    "merger-like": merger_like,
}
