"""Pins of the oracle's interaction test (Sec. 3.1; compare() of Alg. 1-3) against cases whose
answer follows from the geometry by hand."""
import math

import numpy as np
import pytest

import oracle
from tests.cases import seg, segset


def one(q_row, e_row, d, Ts=-1e300, Te=1e300):
    hit, tin, tout, smin = oracle.eval_pairs(segset([e_row]), segset([q_row]), [0], [0], Ts, Te, d)
    return bool(hit[0]), float(tin[0]), float(tout[0]), float(smin[0])


@pytest.mark.parametrize("factor,expect_hit", [(1 - 1e-3, True), (1 + 1e-3, False)])
def test_parallel_constant_separation(factor, expect_hit):
    # Both move with velocity (1,0,0) on [0,10]; separation is s in y for all t.
    d = 5.0
    s = d * factor
    q = seg((0, 0, 0), 0, (10, 0, 0), 10)
    e = seg((0, s, 0), 0, (10, s, 0), 10)
    hit, tin, tout, smin = one(q, e, d)
    assert hit == expect_hit
    assert smin == pytest.approx(s, rel=1e-15)
    if expect_hit:
        assert (tin, tout) == (0.0, 10.0)


def test_parallel_partial_window():
    # Same motion p(t) = (t, s, 0) for the entry, but it only exists on [2, 12]: window [2, 10].
    q = seg((0, 0, 0), 0, (10, 0, 0), 10)
    e = seg((2, 1, 0), 2, (12, 1, 0), 12)
    hit, tin, tout, _ = one(q, e, 2.0)
    assert hit and (tin, tout) == (2.0, 10.0)


def test_head_on():
    # q: -L -> L, e: L -> -L on [0,T]; separation |2L(1 - 2t/T)| <= d on
    # t in [T/2 (1 - d/(2L)), T/2 (1 + d/(2L))] = [7.5, 12.5] for L = 10, T = 20, d = 5.
    L, T, d = 10.0, 20.0, 5.0
    q = seg((-L, 0, 0), 0, (L, 0, 0), T)
    e = seg((L, 0, 0), 0, (-L, 0, 0), T)
    hit, tin, tout, smin = one(q, e, d)
    assert hit
    assert tin == pytest.approx(T / 2 * (1 - d / (2 * L)), abs=1e-12 * T)
    assert tout == pytest.approx(T / 2 * (1 + d / (2 * L)), abs=1e-12 * T)
    assert smin == pytest.approx(0.0, abs=1e-12)


def _perpendicular(h, d, L=10.0, T=20.0):
    # q moves along x from -L to L on [0,T]; e sits at (0, h, 0). sep^2 = x(t)^2 + h^2 with
    # x(t) = -L + 2Lt/T, so the hit is |x| <= sqrt(d^2 - h^2):
    # t in T/2 (1 -+ sqrt(d^2 - h^2) / L).
    q = seg((-L, 0, 0), 0, (L, 0, 0), T)
    e = seg((0, h, 0), 0, (0, h, 0), T)
    return q, e, L, T


def test_perpendicular_tangent_is_single_instant():
    d = 5.0
    q, e, L, T = _perpendicular(d, d)
    hit, tin, tout, smin = one(q, e, d)
    assert hit
    assert tin == tout == pytest.approx(T / 2, abs=1e-12 * T)
    assert smin == pytest.approx(d, rel=1e-15)


@pytest.mark.parametrize("factor", [1 - 1e-6, 1 + 1e-6, 0.5, 0.0])
def test_perpendicular_offsets(factor):
    d = 5.0
    h = d * factor
    q, e, L, T = _perpendicular(h, d)
    hit, tin, tout, smin = one(q, e, d)
    assert smin == pytest.approx(h, rel=1e-12, abs=1e-14)
    if h > d:
        assert not hit
        return
    half = math.sqrt(d * d - h * h) / L
    assert hit
    assert tin == pytest.approx(T / 2 * (1 - half), abs=1e-9 * T)
    assert tout == pytest.approx(T / 2 * (1 + half), abs=1e-9 * T)


def test_stationary_point_query_vs_moving_entry():
    # A zero-length (stationary) query at the origin; the entry passes along y = h: the same
    # geometry as the perpendicular case with the roles swapped (Sec. 2.1's supernova query).
    d, h, L, T = 3.0, 1.0, 4.0, 8.0
    q = seg((0, 0, 0), 0, (0, 0, 0), T)
    e = seg((-L, h, 0), 0, (L, h, 0), T)
    hit, tin, tout, smin = one(q, e, d)
    half = math.sqrt(d * d - h * h) / L
    assert hit
    assert tin == pytest.approx(T / 2 * (1 - half), abs=1e-12 * T)
    assert tout == pytest.approx(T / 2 * (1 + half), abs=1e-12 * T)
    assert smin == pytest.approx(h, rel=1e-14)


def test_disjoint_windows():
    q = seg((0, 0, 0), 0, (1, 0, 0), 1)
    e = seg((0, 0, 0), 2, (1, 0, 0), 3)
    hit, _, _, smin = one(q, e, 10.0)
    assert not hit and math.isinf(smin)


def test_touching_windows_are_not_interactions():
    # Consecutive instants share t = 1 at the same point; the overlap has zero length.
    q = seg((0, 0, 0), 0, (1, 0, 0), 1)
    e = seg((1, 0, 0), 1, (2, 0, 0), 2)
    hit, _, _, smin = one(q, e, 10.0)
    assert not hit and math.isinf(smin)


def test_window_clipped_to_overlap_and_query_interval():
    # Both stationary 1 apart: within d = 2 whenever both exist, i.e. on [5, 10]; with the query
    # interval [6, 8] the interval is [6, 8].
    q = seg((0, 0, 0), 0, (0, 0, 0), 10)
    e = seg((1, 0, 0), 5, (1, 0, 0), 15)
    assert one(q, e, 2.0)[:3] == (True, 5.0, 10.0)
    assert one(q, e, 2.0, Ts=6.0, Te=8.0)[:3] == (True, 6.0, 8.0)
    assert not one(q, e, 2.0, Ts=10.0, Te=12.0)[0]


def test_nearly_equal_velocities_use_the_stable_root():
    # q: y = 0 moving (1,0,0); e: starts at y = D0 = 5 + 2^-30 and drifts with dy/dt = -2^-30.
    # Relative y = -(D0 - delta t) so |y| <= d for t in [(D0-d)/delta, (D0+d)/delta] = [1, ~1e10]
    # clipped to the window [0, 8]. Every input and the velocity are exact binary fractions.
    # The textbook root (-b - sqrt(disc))/a loses ~3e-7 of t_in here (cancellation); the stable
    # pair s/a, c/s is accurate to ~1e-10.
    delta = 2.0 ** -30
    D0 = 5.0 + delta
    q = seg((0, 0, 0), 0, (8, 0, 0), 8)
    e = seg((0, D0, 0), 0, (8, D0 - 8 * delta, 0), 8)
    hit, tin, tout, _ = one(q, e, 5.0)
    assert hit
    assert tin == pytest.approx(1.0, abs=1e-9 * 8)
    assert tout == 8.0


def test_swap_symmetry():
    rng = np.random.default_rng(7)
    from tests.cases import random_segments
    a = random_segments(rng, 60)
    b = random_segments(rng, 60)
    qi, ei = np.meshgrid(np.arange(60), np.arange(60), indexing="ij")
    qi, ei = qi.ravel(), ei.ravel()
    h1, i1, o1, s1 = oracle.eval_pairs(b, a, qi, ei, -1e300, 1e300, 2.5)
    h2, i2, o2, s2 = oracle.eval_pairs(a, b, ei, qi, -1e300, 1e300, 2.5)
    assert h1.sum() > 20
    np.testing.assert_array_equal(h1, h2)
    np.testing.assert_allclose(i1[h1], i2[h2], rtol=0, atol=1e-12)
    np.testing.assert_allclose(o1[h1], o2[h2], rtol=0, atol=1e-12)


def test_translation_invariance():
    rng = np.random.default_rng(11)
    from tests.cases import random_segments
    from paper_1410_2698_gb300.workloads import Segments
    a = random_segments(rng, 50)
    b = random_segments(rng, 50)
    off = np.array([1e3, -1e3, 5e2, 0, 1e3, -1e3, 5e2, 0])
    a2 = Segments.from_matrix(a.as_matrix() + off)
    b2 = Segments.from_matrix(b.as_matrix() + off)
    qi, ei = np.meshgrid(np.arange(50), np.arange(50), indexing="ij")
    qi, ei = qi.ravel(), ei.ravel()
    h1, i1, o1, s1 = oracle.eval_pairs(b, a, qi, ei, -1e300, 1e300, 3.0)
    h2, i2, o2, s2 = oracle.eval_pairs(b2, a2, qi, ei, -1e300, 1e300, 3.0)
    keep = np.abs(s1 - 3.0) > 1e-9 * 3.0
    np.testing.assert_array_equal(h1[keep], h2[keep])
    both = h1 & h2
    np.testing.assert_allclose(i1[both], i2[both], atol=1e-9 * 3.0)
    np.testing.assert_allclose(o1[both], o2[both], atol=1e-9 * 3.0)
