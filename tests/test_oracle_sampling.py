"""Pins of the oracle against dense time sampling of the separation (a brute-force reading of the
problem of Sec. 3.1), and of its temporal pruning against the plain all-pairs loop."""
import numpy as np
import pytest

import oracle
from tests.cases import random_segments, sample_separation


def _all_pairs(nq, ne):
    qi, ei = np.meshgrid(np.arange(nq), np.arange(ne), indexing="ij")
    return qi.ravel(), ei.ravel()


@pytest.mark.parametrize("seed,d,stationary", [(1, 1.5, 0.0), (2, 3.0, 0.2), (3, 1.2, 0.5)])
def test_dense_time_sampling(seed, d, stationary):
    rng = np.random.default_rng(seed)
    q = random_segments(rng, 40, stationary_frac=stationary)
    e = random_segments(rng, 120, stationary_frac=stationary)
    Ts, Te = 1.0, 11.0
    qi, ei = _all_pairs(q.n, e.n)
    hit, tin, tout, smin = oracle.eval_pairs(e, q, qi, ei, Ts, Te, d)
    t_lo = np.maximum(np.maximum(q.t0[qi], e.t0[ei]), Ts)
    t_hi = np.minimum(np.minimum(q.t1[qi], e.t1[ei]), Te)
    live = t_lo < t_hi
    assert hit.sum() >= 10 and (live & ~hit).sum() >= 10
    assert not np.any(hit & ~live)
    ns = 20001
    u = np.linspace(0.0, 1.0, ns)
    for k in np.nonzero(live)[0]:
        T = t_hi[k] - t_lo[k]
        t = t_lo[k] + u * T
        s = sample_separation(q, e, np.full(ns, qi[k]), np.full(ns, ei[k]), t)
        # the oracle's minimum separation is a lower bound of every sample and close to the
        # sampled minimum (the sampled distance is Lipschitz in t with the relative speed)
        speed = np.abs(np.diff(s)).max() / (u[1] * T) if T > 0 else 0.0
        assert smin[k] <= s.min() * (1 + 1e-12) + 1e-12
        assert smin[k] >= s.min() - speed * u[1] * T - 1e-12
        if hit[k]:
            assert t_lo[k] <= tin[k] <= tout[k] <= t_hi[k]
            inside = (t >= tin[k]) & (t <= tout[k])
            assert np.all(s[inside] <= d * (1 + 1e-9))
            assert np.all(s[~inside] > d * (1 - 1e-9))
            # interior endpoints are crossings of the threshold: root accuracy by bisection
            for tr in (tin[k], tout[k]):
                if t_lo[k] < tr < t_hi[k]:
                    sr = sample_separation(q, e, np.array([qi[k]]), np.array([ei[k]]),
                                           np.array([tr]))[0]
                    assert abs(sr - d) <= 1e-9 * d + 1e-12 * T * max(speed, 1.0)
        else:
            assert s.min() > d * (1 - 1e-9)


def test_temporal_pruning_equals_all_pairs():
    rng = np.random.default_rng(5)
    q = random_segments(rng, 70, t_range=(0, 30))
    e = random_segments(rng, 400, t_range=(0, 30))
    Ts, Te, d = 3.0, 25.0, 2.0
    res = oracle.search(e, q, Ts, Te, d)
    qi, ei = _all_pairs(q.n, e.n)
    hit, tin, tout, _ = oracle.eval_pairs(e, q, qi, ei, Ts, Te, d)
    assert hit.sum() > 50
    np.testing.assert_array_equal(res["q_idx"], qi[hit])
    np.testing.assert_array_equal(res["e_idx"], ei[hit])
    np.testing.assert_array_equal(res["t_in"], tin[hit])
    np.testing.assert_array_equal(res["t_out"], tout[hit])
    # the window test runs on every pair whose time extents can overlap the clipped window
    t_lo = np.maximum(np.maximum(q.t0[qi], e.t0[ei]), Ts)
    t_hi = np.minimum(np.minimum(q.t1[qi], e.t1[ei]), Te)
    assert res["n_tests"] >= int((t_lo < t_hi).sum())
    assert res["n_tests"] < qi.size


def test_counting_baseline_matches_search():
    rng = np.random.default_rng(9)
    q = random_segments(rng, 90, t_range=(0, 20))
    e = random_segments(rng, 500, t_range=(0, 20))
    res = oracle.search(e, q, 0.0, 20.0, 1.5)
    for threads in (1, 3):
        hits, tests, qsegs = oracle.search_count(e, q, 0.0, 20.0, 1.5, threads=threads)
        assert hits == res["q_idx"].size
        assert tests == res["n_tests"]
        assert qsegs == q.n


def test_multithreaded_search_equals_single_threaded():
    """The two-pass multithreaded search (counts, prefix sum, rows at offsets) returns exactly the
    single-threaded search's rows and test count, for several thread counts."""
    rng = np.random.default_rng(13)
    q = random_segments(rng, 120, t_range=(0, 25))
    e = random_segments(rng, 700, t_range=(0, 25))
    ref = oracle.search(e, q, 2.0, 22.0, 1.8, threads=1)
    assert ref["q_idx"].size > 50
    for threads in (2, 5):
        got = oracle.search(e, q, 2.0, 22.0, 1.8, threads=threads)
        for k in ("q_idx", "e_idx", "t_in", "t_out", "s_min"):
            np.testing.assert_array_equal(got[k], ref[k])
        assert got["n_tests"] == ref["n_tests"]
    empty = oracle.search(e, q, 40.0, 50.0, 1.8, threads=3)  # no window overlaps
    assert empty["q_idx"].size == 0 and empty["n_tests"] == 0
