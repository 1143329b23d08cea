"""The GPU exact test against the closed-form cases that pin the oracle (each expected value
derived by hand from the geometry, as in tests/test_oracle_analytic.py), through every index, and
element by element against the oracle's evaluation of the same pairs. The GPU decides hits
without division (the minimum of the distance quadratic over the window) and computes the roots
with fused multiply-adds and refined reciprocal / square-root estimates, so it faces these cases
directly rather than through the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api
from paper_1410_2698_gb300.workloads import Segments
from tests import parity
from tests.cases import random_segments, seg, segset

pytestmark = pytest.mark.gpu

KINDS = ("brute", "temporal", "spatiotemporal", "spatial")


def _gpu_rows(q, e, d, Ts=-1e9, Te=1e9, kind="brute"):
    idx = api.ts_build_index(e, kind=kind)
    try:
        return api.ts_search(idx, q, d, Ts, Te).to_host(sort=True)
    finally:
        idx.free()


def _one(q_row, e_row, d, Ts=-1e9, Te=1e9):
    """The single pair's GPU result through every index: (hit, t_in, t_out), the same for all."""
    out = None
    for kind in KINDS:
        r = _gpu_rows(segset([q_row]), segset([e_row]), d, Ts, Te, kind)
        got = (r["q_idx"].size == 1, float(r["t_in"][0]) if r["t_in"].size else None,
               float(r["t_out"][0]) if r["t_out"].size else None)
        assert r["q_idx"].size <= 1, kind
        if out is None:
            out = got
        assert got == out, (kind, got, out)
    return out


def test_nearly_equal_velocities_use_the_stable_root():
    # relative y = -(D0 - delta t) with D0 = 5 + 2^-30, delta = 2^-30: |y| <= 5 for t >= 1
    delta = 2.0 ** -30
    D0 = 5.0 + delta
    q = seg((0, 0, 0), 0, (8, 0, 0), 8)
    e = seg((0, D0, 0), 0, (8, D0 - 8 * delta, 0), 8)
    hit, tin, tout = _one(q, e, 5.0)
    assert hit
    assert abs(tin - 1.0) <= 1e-9 * 8
    assert tout == 8.0


@pytest.mark.parametrize("factor", [1 - 1e-6, 1 + 1e-6, 0.5, 0.0])
def test_perpendicular_offsets(factor):
    # q along x from -10 to 10 on [0, 20]; e fixed at (0, h, 0): hit iff h <= d, on
    # t in 10 (1 -+ sqrt(d^2 - h^2) / 10)
    d = 5.0
    h = d * factor
    q = seg((-10, 0, 0), 0, (10, 0, 0), 20)
    e = seg((0, h, 0), 0, (0, h, 0), 20)
    hit, tin, tout = _one(q, e, d)
    if h > d:
        assert not hit
        return
    half = math.sqrt(d * d - h * h) / 10.0
    assert hit
    assert abs(tin - 10 * (1 - half)) <= 1e-9 * 20
    assert abs(tout - 10 * (1 + half)) <= 1e-9 * 20


def test_tangent_is_a_single_instant():
    hit, tin, tout = _one(seg((-10, 0, 0), 0, (10, 0, 0), 20), seg((0, 5, 0), 0, (0, 5, 0), 20),
                          5.0)
    assert hit and abs(tin - 10.0) <= 1e-9 * 20 and abs(tout - 10.0) <= 1e-9 * 20


def test_partially_overlapping_windows_are_clipped():
    # the entry follows (t, 1, 0) on [2, 12]; the query (t, 0, 0) on [0, 10]: window [2, 10]
    assert _one(seg((0, 0, 0), 0, (10, 0, 0), 10), seg((2, 1, 0), 2, (12, 1, 0), 12), 2.0) == \
        (True, 2.0, 10.0)
    # both stationary 1 apart: [5, 10] by the segments, [6, 8] by the query interval
    q, e = seg((0, 0, 0), 0, (0, 0, 0), 10), seg((1, 0, 0), 5, (1, 0, 0), 15)
    assert _one(q, e, 2.0) == (True, 5.0, 10.0)
    assert _one(q, e, 2.0, Ts=6.0, Te=8.0) == (True, 6.0, 8.0)
    assert not _one(q, e, 2.0, Ts=10.0, Te=12.0)[0]


def test_stationary_query_and_touching_windows():
    d, h, L, T = 3.0, 1.0, 4.0, 8.0
    hit, tin, tout = _one(seg((0, 0, 0), 0, (0, 0, 0), T), seg((-L, h, 0), 0, (L, h, 0), T), d)
    half = math.sqrt(d * d - h * h) / L
    assert hit and abs(tin - T / 2 * (1 - half)) <= 1e-9 * T
    assert abs(tout - T / 2 * (1 + half)) <= 1e-9 * T
    # consecutive instants sharing t = 1 at the same point: no positive overlap, no hit
    assert not _one(seg((0, 0, 0), 0, (1, 0, 0), 1), seg((1, 0, 0), 1, (2, 0, 0), 2), 10.0)[0]


def _all_pairs(q, e, d, kind):
    return _gpu_rows(q, e, d, -1e9, 1e9, kind)


def test_swap_symmetry():
    # searching A against B and B against A gives the same pairs with the same intervals
    rng = np.random.default_rng(7)
    a = random_segments(rng, 60)
    b = random_segments(rng, 60)
    for kind in KINDS:
        ab = _all_pairs(a, b, 2.5, kind)
        ba = _all_pairs(b, a, 2.5, kind)
        assert ab["q_idx"].size > 20
        order = np.lexsort((ba["q_idx"], ba["e_idx"]))
        np.testing.assert_array_equal(ab["q_idx"], ba["e_idx"][order])
        np.testing.assert_array_equal(ab["e_idx"], ba["q_idx"][order])
        np.testing.assert_allclose(ab["t_in"], ba["t_in"][order], rtol=0, atol=1e-12)
        np.testing.assert_allclose(ab["t_out"], ba["t_out"][order], rtol=0, atol=1e-12)


def test_translation_by_a_large_offset():
    rng = np.random.default_rng(11)
    a = random_segments(rng, 50)
    b = random_segments(rng, 50)
    off = np.array([1e3, -1e3, 5e2, 0, 1e3, -1e3, 5e2, 0])
    a2 = Segments.from_matrix(a.as_matrix() + off)
    b2 = Segments.from_matrix(b.as_matrix() + off)
    d = 3.0
    for kind in KINDS:
        r1 = _all_pairs(a, b, d, kind)
        r2 = _all_pairs(a2, b2, d, kind)
        # both against the oracle of their own coordinates
        parity.compare(r1, oracle.search(b, a, -1e9, 1e9, d), b, a, -1e9, 1e9, d)
        parity.compare(r2, oracle.search(b2, a2, -1e9, 1e9, d), b2, a2, -1e9, 1e9, d)
        # and the same pairs (away from tangency) and intervals as the untranslated search
        _, _, _, smin = oracle.eval_pairs(b, a, r1["q_idx"], r1["e_idx"], -1e9, 1e9, d)
        keep = np.abs(smin - d) > 1e-9 * d
        k1 = (r1["q_idx"].astype(np.int64) << 32) | r1["e_idx"]
        k2 = (r2["q_idx"].astype(np.int64) << 32) | r2["e_idx"]
        common, i1, i2 = np.intersect1d(k1, k2, return_indices=True)
        assert set(k1[keep]) <= set(common.tolist())
        np.testing.assert_allclose(r1["t_in"][i1], r2["t_in"][i2], atol=1e-9 * d)
        np.testing.assert_allclose(r1["t_out"][i1], r2["t_out"][i2], atol=1e-9 * d)


def test_every_pair_against_the_oracle_element_by_element():
    # the GPU's decision and interval for every (query, entry) pair of two small random sets,
    # against oracle.eval_pairs of the same pairs (brute force: every pair is a candidate)
    rng = np.random.default_rng(5)
    a = random_segments(rng, 120, stationary_frac=0.2)
    b = random_segments(rng, 150, stationary_frac=0.2)
    d = 2.0
    got = _all_pairs(a, b, d, "brute")
    qi, ei = np.meshgrid(np.arange(a.n), np.arange(b.n), indexing="ij")
    qi, ei = qi.ravel(), ei.ravel()
    hit, tin, tout, smin = oracle.eval_pairs(b, a, qi, ei, -1e9, 1e9, d)
    key = (qi.astype(np.int64) << 32) | ei
    gk = (got["q_idx"].astype(np.int64) << 32) | got["e_idx"]
    gpu_hit = np.isin(key, gk)
    differ = gpu_hit != hit
    assert not np.any(differ & (np.abs(smin - d) > 1e-9 * d))
    assert hit.sum() > 50
    both = np.nonzero(gpu_hit & hit)[0]
    pos = np.searchsorted(gk, key[both])
    T = parity.overlap_duration(b, a, qi[both], ei[both], -1e9, 1e9)
    assert np.all(np.abs(got["t_in"][pos] - tin[both]) <= 1e-9 * T)
    assert np.all(np.abs(got["t_out"][pos] - tout[both]) <= 1e-9 * T)
