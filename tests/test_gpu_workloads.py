"""GPU parity at the benchmark workloads' sizes: the Random-walk 1M configuration in full (the
oracle's temporal pruning finishes it in seconds), and the dense and merger-like configurations
on seeded samples of query trajectories."""
import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rw1m():
    return workloads.random_walk_1m()


@pytest.fixture(scope="module")
def rw1m_indexes(rw1m):
    out = {k: api.ts_build_index(rw1m.db, kind=k)
           for k in ("temporal", "spatiotemporal", "spatial")}
    yield out
    for idx in out.values():
        idx.free()


@pytest.mark.parametrize("d", [1.0, 5.0, 10.0, 25.0])
def test_random_walk_1m_full(rw1m, rw1m_indexes, d):
    ref = oracle.search(rw1m.db, rw1m.queries, rw1m.t_start, rw1m.t_end, d)
    counts = {}
    for kind, idx in rw1m_indexes.items():
        got = api.ts_search(idx, rw1m.queries, d, rw1m.t_start, rw1m.t_end).to_host(sort=True)
        parity.compare(got, ref, rw1m.db, rw1m.queries, rw1m.t_start, rw1m.t_end, d)
        counts[kind] = got["q_idx"].size
    # every query segment meets its own database twin over its whole extent
    assert ref["q_idx"].size >= rw1m.queries.n


def _trajectory_sample(w, n_traj, seed):
    seg_per = w.queries.n // len(w.query_traj_ids)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(w.query_traj_ids), size=n_traj, replace=False))
    idx = (pick[:, None] * seg_per + np.arange(seg_per)[None, :]).ravel()
    return w.queries.take(idx)


@pytest.fixture(scope="module")
def dense_small():
    # the dense configuration's density (20,000 trajectories x 101 samples in [0,50]^3)
    return workloads.dense()


@pytest.mark.parametrize("d", [0.5, 2.0])
def test_dense_sampled(dense_small, d):
    w = dense_small
    q = _trajectory_sample(w, 6, seed=7)
    ref = oracle.search(w.db, q, w.t_start, w.t_end, d)
    for kind in ("temporal", "spatiotemporal", "spatial"):
        idx = api.ts_build_index(w.db, kind=kind)
        got = api.ts_search(idx, q, d, w.t_start, w.t_end).to_host(sort=True)
        parity.compare(got, ref, w.db, q, w.t_start, w.t_end, d)
        idx.free()
    assert ref["q_idx"].size > q.n  # dense: more than the self matches
