"""Pins of the oracle's index structures and schedules: the paper's worked examples (Fig.
example_index of Sec. 4.2, Fig. spatiotemporal_indexing of Sec. 4.3) and hand-derived cases."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_temporal_index_worked_example():
    g = _golden("temporal_index_example.json")
    seg = np.array(g["segments_t_start_t_end"])
    ti = oracle.temporal_index(seg[:, 0], seg[:, 1], g["m"])
    exp = g["expected"]
    np.testing.assert_array_equal(ti["perm"], np.arange(15))
    np.testing.assert_array_equal(ti["bin_start"], exp["bin_start"])
    np.testing.assert_array_equal(ti["bin_end"], exp["bin_end"])
    np.testing.assert_array_equal(ti["bin_off"][:-1], exp["bin_first"])
    np.testing.assert_array_equal(ti["bin_off"][1:] - 1, exp["bin_last"])
    assert ti["tmin"] == 0.0 and ti["b"] == 3.0


def test_temporal_index_sorts_by_start_time_with_stable_ties():
    t0 = np.array([5.0, 1.0, 3.0, 1.0, 0.0, 5.0])
    t1 = t0 + 1.0
    ti = oracle.temporal_index(t0, t1, 2)
    # sorted by t0, equal t0 in original order
    np.testing.assert_array_equal(ti["perm"], [4, 1, 3, 2, 0, 5])
    # t_min = 0, t_max = 6, b = 3: bins [0,3) and [3,6]
    np.testing.assert_array_equal(ti["bin_of"], [0, 0, 0, 1, 1, 1])
    np.testing.assert_array_equal(ti["bin_end"], [3.0, 6.0])


def test_temporal_schedule_worked_example():
    g = _golden("temporal_index_example.json")
    seg = np.array(g["segments_t_start_t_end"])
    ti = oracle.temporal_index(seg[:, 0], seg[:, 1], g["m"])
    # bins (start, end): (0,7.5) (3,6.2) (6,11) (9,12); offsets 0,6,9,12,15
    w0 = np.array([0.5, 6.5, 7.6, 11.95, 12.0, 2.0, 6.2])
    w1 = np.array([1.0, 7.0, 8.0, 12.0, 13.0, 3.0, 6.3])
    lo, hi = oracle.temporal_schedule(ti, w0, w1)
    # [0.5,1]: bins 0..0 -> [0,6)
    # [6.5,7]: first bin ending after 6.5 is B_0 (7.5); last starting before 7 is B_2 -> [0,12)
    # [7.6,8]: B_0 ends 7.5, B_1 6.2, B_2 11 -> from B_2; last start before 8 is B_2 -> [9,12)
    # [11.95,12]: B_2 ends 11 <= 11.95, B_3 ends 12 -> from B_3 to B_3 -> [12,15)
    # [12,13]: no bin ends after 12 -> empty
    # [2,3]: B_0..B_0 (B_1 starts at 3, not before 3) -> [0,6)
    # [6.2,6.3]: B_0 (7.5 > 6.2) .. B_2 (6 < 6.3) -> [0,12)
    np.testing.assert_array_equal(lo, [0, 0, 9, 12, 0, 0, 0])
    np.testing.assert_array_equal(hi, [6, 12, 12, 15, 0, 6, 12])


def _st_example():
    g = _golden("spatiotemporal_x_example.json")
    ep = np.array(g["endpoints"], dtype=np.float64)  # (10, 2, 3)
    emin = ep.min(axis=1)
    emax = ep.max(axis=1)
    return g, emin, emax


def test_spatiotemporal_x_array_worked_example():
    g, emin, emax = _st_example()
    m, v = g["m"], g["v"]
    ids, off = oracle.st_dim(emin[:, 0], emax[:, 0], g["bin_of"], m, g["x_lo"], g["x_w"], v)
    np.testing.assert_array_equal(ids, g["expected_X"])
    for key, rng in g["expected_X_ranges_by_bin_then_subbin"].items():
        i, j = map(int, key.split(","))
        a, b = off[j * m + i], off[j * m + i + 1]
        if rng is None:
            assert a == b
        else:
            assert (a, b - 1) == tuple(rng)


def test_st_params_respect_longest_segment():
    # extent [0, 10], longest segment 3 -> at most floor(10/3) = 3 subbins of width 10/3
    emin = np.array([0.0, 2.0, 7.0])
    emax = np.array([1.0, 5.0, 10.0])
    assert oracle.st_params(emin, emax, 8) == (0.0, 10.0 / 3.0, 3)
    assert oracle.st_params(emin, emax, 2) == (0.0, 5.0, 2)
    # all points equal: one subbin
    assert oracle.st_params(np.ones(3), np.ones(3), 4)[2] == 1


def test_st_schedule_hand_case():
    # The example geometry of Fig. spatiotemporal_indexing with x, y subbins of width 4 and z
    # subbins of width 5 (origin 0), bins B_0 = l0..l3, B_1 = l4..l7, B_2 = l8..l9.
    g, emin, emax = _st_example()
    m, v = 3, 3
    bin_of = np.array(g["bin_of"])
    tidx = {"bin_start": np.array([0.0, 1.0, 2.0]), "bin_end": np.array([1.0, 2.0, 3.0]),
            "bin_off": np.array([0, 4, 8, 10], dtype=np.int64)}
    dims = []
    for dim, w in zip(range(3), (4.0, 4.0, 5.0)):
        ids, off = oracle.st_dim(emin[:, dim], emax[:, dim], bin_of, m, 0.0, w, v)
        dims.append({"lo": 0.0, "w": w, "v": v, "off": off, "ids": ids})
    # Query A: time window inside B_0..B_1, x in [1, 2] (d-expanded [0.5, 2.5]: x subbin 0 only),
    # y in [3, 5] and z in [4, 6] (two subbins each). Only x qualifies; subbin 0 over bins 0..1
    # holds X[0..3] = l1, l3, l4, l5.
    # Query B: same window, x in [1, 6] (two subbins), y in [9, 10] (subbin 2 only: ids of
    # B_{0,2}, B_{1,2} = l6), z in [11, 12] (subbin 2 only: l6 in B_1). Tie of one id each ->
    # lowest dimension, y.
    # Query C: x over two subbins, y over two, z over two -> temporal fallback [0, 8).
    # Query D: window after all bins -> empty temporal range.
    # Query E: x in [-30, -20] (d-expanded below every subbin): no entry can be near -> empty
    # range in x.
    qmin = [np.array([1.0, 1.0, 1.0, 1.0, -30.0]), np.array([3.0, 9.0, 3.0, 3.0, 3.0]),
            np.array([4.0, 11.0, 4.0, 4.0, 4.0])]
    qmax = [np.array([2.0, 6.0, 6.0, 2.0, -20.0]), np.array([5.0, 10.0, 5.0, 5.0, 5.0]),
            np.array([6.0, 12.0, 6.0, 6.0, 6.0])]
    w0 = np.array([0.5, 0.5, 0.5, 3.5, 0.5])
    w1 = np.array([1.5, 1.5, 1.5, 4.0, 1.5])
    sel, lo, hi = oracle.st_schedule(tidx, dims, qmin, qmax, w0, w1, 0.5)
    assert (sel[0], lo[0], hi[0]) == (0, 0, 4)
    np.testing.assert_array_equal(dims[0]["ids"][lo[0]:hi[0]], [1, 3, 4, 5])
    assert sel[1] == 1
    np.testing.assert_array_equal(dims[1]["ids"][lo[1]:hi[1]], [6])
    assert (sel[2], lo[2], hi[2]) == (3, 0, 8)
    assert (sel[3], lo[3], hi[3]) == (3, 0, 0)
    assert sel[4] == 0 and lo[4] == hi[4]


def test_fsg_hand_case():
    # g = 2 cells per dimension over [0,2]^3 (origin 0, width 1). Entry 0 spans x 0.5..1.5 (cells
    # x 0 and 1), entry 1 sits in cell (0,0,0), entry 2 in cell (1,1,1).
    emin = np.array([[0.5, 0.2, 0.2], [0.0, 0.0, 0.0], [1.5, 1.5, 1.5]])
    emax = np.array([[1.5, 0.4, 0.4], [0.2, 0.2, 0.2], [2.0, 2.0, 2.0]])
    lo, w = zip(*[oracle.grid_params(emin[:, k], emax[:, k], 2) for k in range(3)])
    assert lo == (0.0, 0.0, 0.0) and w == (1.0, 1.0, 1.0)
    A, off = oracle.fsg([emin[:, k] for k in range(3)], [emax[:, k] for k in range(3)], 2, lo, w)
    # h = (cx*2 + cy)*2 + cz: entry 0 in h = 0 and h = 4; entry 1 in h = 0; entry 2 in h = 7.
    np.testing.assert_array_equal(A, [0, 1, 0, 2])
    np.testing.assert_array_equal(off, [0, 2, 2, 2, 2, 3, 3, 3, 4])
    # A query box covering the whole grid meets entry 0 twice (cells 0 and 4) but keeps it once.
    qmin = [np.array([0.0]), np.array([0.0]), np.array([0.0])]
    qmax = [np.array([2.0]), np.array([2.0]), np.array([2.0])]
    raw, uniq = oracle.fsg_candidates([emin[:, k] for k in range(3)],
                                      [emax[:, k] for k in range(3)], 2, lo, w, A, off, qmin,
                                      qmax, 0.1)
    assert (raw[0], uniq[0]) == (4, 3)
    # A query in cell (1,0,0) only (x 1.2..1.3, y,z 0.1..0.2, d = 0.05) meets entry 0 once.
    raw, uniq = oracle.fsg_candidates([emin[:, k] for k in range(3)],
                                      [emax[:, k] for k in range(3)], 2, lo, w, A, off,
                                      [np.array([1.2]), np.array([0.1]), np.array([0.1])],
                                      [np.array([1.3]), np.array([0.2]), np.array([0.2])], 0.05)
    assert (raw[0], uniq[0]) == (1, 1)


def test_one_cell_grid_hand_case():
    # g = 2 over [0,2]^3 (origin 0, width 1). Minimum corners: entry 0 (0.5, 0.2, 0.2) -> cell 0,
    # entry 1 (0, 0, 0) -> cell 0, entry 2 (1.5, 1.5, 1.5) -> cell (1,1,1) = 7.
    emin = np.array([[0.5, 0.2, 0.2], [0.0, 0.0, 0.0], [1.5, 1.5, 1.5]])
    emax = np.array([[1.5, 0.4, 0.4], [0.2, 0.2, 0.2], [2.0, 2.0, 2.0]])
    lo, w = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    A, off = oracle.grid1([emin[:, k] for k in range(3)], 2, lo, w)
    np.testing.assert_array_equal(A, [0, 1, 2])
    np.testing.assert_array_equal(off, [0, 2, 2, 2, 2, 2, 2, 2, 3])
    longest = emax.max(axis=0) - 0  # per-axis largest extent: x 1.0 (entry 0), y and z 0.5
    longest = (emax - emin).max(axis=0)
    assert tuple(longest) == (1.0, 0.5, 0.5)
    # query MBB x 1.2..1.3, y and z 0.1..0.2, d = 0.05: minimum corners of entries within d lie in
    # x [0.15, 1.35] (cells 0..1), y and z [-0.45, 0.25] (cell 0): runs (0,0) and (1,0), the z-run
    # cells (0,0,0) with 2 entries and (1,0,0) with none.
    runs, cand = oracle.grid1_candidates(2, lo, w, longest, off, [np.array([1.2]),
                                         np.array([0.1]), np.array([0.1])],
                                         [np.array([1.3]), np.array([0.2]), np.array([0.2])],
                                         np.array([0.0]), np.array([1.0]), 0.05)
    assert (runs[0], cand[0]) == (2, 2)
    # an empty window gives no candidates
    runs, cand = oracle.grid1_candidates(2, lo, w, longest, off, [np.array([1.2])] * 3,
                                         [np.array([1.3])] * 3, np.array([1.0]),
                                         np.array([1.0]), 0.05)
    assert (runs[0], cand[0]) == (0, 0)


def test_one_cell_grid_candidates_cover_every_hit():
    # every pair within d must be a candidate of the grid schedule (checked against the search)
    from tests.cases import random_segments
    rng = np.random.default_rng(21)
    db = random_segments(rng, 400, box=20.0, max_len=2.0)
    q = random_segments(rng, 60, box=20.0, max_len=2.0)
    d = 1.5
    emin = [np.minimum(db.x0, db.x1), np.minimum(db.y0, db.y1), np.minimum(db.z0, db.z1)]
    emax = [np.maximum(db.x0, db.x1), np.maximum(db.y0, db.y1), np.maximum(db.z0, db.z1)]
    g = 7
    lo, w = zip(*[oracle.grid_params(emin[k], emax[k], g) for k in range(3)])
    longest = [float((emax[k] - emin[k]).max()) for k in range(3)]
    A, off = oracle.grid1(emin, g, lo, w)
    res = oracle.search(db, q, -1e9, 1e9, d)
    cell = {}
    for pos, s in enumerate(A):
        h = int(np.searchsorted(off, pos, side="right") - 1)
        cell[int(s)] = h
    qmin = [np.minimum(q.x0, q.x1), np.minimum(q.y0, q.y1), np.minimum(q.z0, q.z1)]
    qmax = [np.maximum(q.x0, q.x1), np.maximum(q.y0, q.y1), np.maximum(q.z0, q.z1)]
    for qi, ei in zip(res["q_idx"], res["e_idx"]):
        h = cell[int(ei)]
        c = (h // (g * g), (h // g) % g, h % g)
        for k in range(3):
            a = (qmin[k][qi] - d) - longest[k]
            b = qmax[k][qi] + d
            assert lo[k] + c[k] * w[k] <= b and (c[k] == g - 1 or lo[k] + (c[k] + 1) * w[k] > a)


def test_st_schedule_widens_an_expanded_extent_that_lands_on_a_boundary():
    # x subbins [0,10), [10,20), [20,30), [30,inf) (lo 0, width 10); y and z subbins of width 1,
    # so a query with d = 2 meets at least four of them there and only x can serve it.
    # Query A: x in [12, 12.5]: the d-expanded extent starts exactly at the boundary 10, the
    # relative widening of the extent (reading: a relative 1e-12, against the rounding of
    # min - d) makes it meet [0,10) as well as [10,20): two subbins, so the temporal range
    # serves it (selector 3). Query B: x in [12.5, 13] starts at 10.5, inside [10,20) only: the
    # x subbin serves it (selector 0) with the ids of subbin 1 in bin 0.
    xs = np.array([5.0, 9.5, 15.0, 25.0, 35.0])
    emin = np.stack([xs, np.full(5, 20.0), np.full(5, 20.0)], axis=1)
    emax = emin.copy()
    bin_of = np.zeros(5, dtype=np.int32)
    tidx = {"bin_start": np.array([0.0]), "bin_end": np.array([1.0]),
            "bin_off": np.array([0, 5], dtype=np.int64)}
    dims = []
    for dim, (w, v) in enumerate([(10.0, 4), (1.0, 40), (1.0, 40)]):
        ids, off = oracle.st_dim(emin[:, dim], emax[:, dim], bin_of, 1, 0.0, w, v)
        dims.append({"lo": 0.0, "w": w, "v": v, "off": off, "ids": ids})
    qmin = [np.array([12.0, 12.5]), np.array([20.0, 20.0]), np.array([20.0, 20.0])]
    qmax = [np.array([12.5, 13.0]), np.array([20.0, 20.0]), np.array([20.0, 20.0])]
    w0, w1 = np.array([0.0, 0.0]), np.array([1.0, 1.0])
    sel, lo, hi = oracle.st_schedule(tidx, dims, qmin, qmax, w0, w1, 2.0)
    assert sel[0] == 3 and (lo[0], hi[0]) == (0, 5)
    assert sel[1] == 0
    np.testing.assert_array_equal(dims[0]["ids"][lo[1]:hi[1]], [2])  # the entry at x = 15
