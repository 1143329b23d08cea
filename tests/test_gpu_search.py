"""GPU parity: the CUDA path through the C ABI against the oracle, on seeded inputs."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads
from paper_1410_2698_gb300.workloads import Segments
from tests import parity
from tests.cases import seg, segset

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny():
    return workloads.tiny()


def _run(db, q, kind, d, Ts, Te, **kw):
    idx = api.ts_build_index(db, kind=kind, **kw)
    res = api.ts_search(idx, q, d, Ts, Te)
    got = res.to_host(sort=True)
    stats = res.stats
    info = idx.info()
    res.free()
    idx.free()
    return got, stats, info


@pytest.mark.parametrize("kind,kw", [
    ("brute", {}),
    ("temporal", {}),
    ("temporal", {"t_bins": 1}),
    ("temporal", {"t_bins": 37}),
    ("temporal", {"t_bins": 20000}),
    ("spatiotemporal", {}),
    ("spatiotemporal", {"sub_bins": 1}),
    ("spatiotemporal", {"sub_bins": 3, "t_bins": 11}),
    ("spatiotemporal", {"sub_bins": 64}),
    ("spatial", {}),
    ("spatial", {"grid_cells": 1}),
    ("spatial", {"grid_cells": 7}),
    ("spatial", {"grid_cells": 100}),
])
def test_tiny_config_matches_oracle(tiny, kind, kw):
    d = tiny.distances[0]
    ref = oracle.search(tiny.db, tiny.queries, tiny.t_start, tiny.t_end, d)
    got, stats, _ = _run(tiny.db, tiny.queries, kind, d, tiny.t_start, tiny.t_end, **kw)
    diag = parity.compare(got, ref, tiny.db, tiny.queries, tiny.t_start, tiny.t_end, d)
    assert diag["rows"] > 1000
    assert stats["n_hits"] == got["q_idx"].size
    assert stats["n_qsegs"] == 2000 - int(np.sum(np.minimum(tiny.queries.t1, tiny.t_end)
                                                 <= np.maximum(tiny.queries.t0, tiny.t_start)))
    assert stats["n_exact"] <= stats["n_tests"]
    if kind == "brute":
        assert stats["n_tests"] == stats["n_qsegs"] * tiny.db.n


def test_well_conditioned_intervals_agree_with_the_oracle_to_rounding(tiny):
    """The kernel's evaluation (fused multiply-adds, refined reciprocal and square root) differs
    from the oracle's plain one only in rounding: for every pair whose minimum separation is not
    within 1e-6 * d of d (roots far from coalescing), both interval ends agree to 1e-11 of the
    pair's overlap, a hundred times inside the acceptance tolerance."""
    d = 5.0
    ref = oracle.search(tiny.db, tiny.queries, tiny.t_start, tiny.t_end, d)
    got, _, _ = _run(tiny.db, tiny.queries, "temporal", d, tiny.t_start, tiny.t_end)
    parity.compare(got, ref, tiny.db, tiny.queries, tiny.t_start, tiny.t_end, d)
    kg = (got["q_idx"].astype(np.int64) << 32) | got["e_idx"].astype(np.int64)
    kr = (ref["q_idx"].astype(np.int64) << 32) | ref["e_idx"].astype(np.int64)
    common, ig, ir = np.intersect1d(kg, kr, return_indices=True)
    well = np.abs(ref["s_min"][ir] - d) > 1e-6 * d
    assert well.sum() > 1000
    T = parity.overlap_duration(tiny.db, tiny.queries, ref["q_idx"][ir].astype(np.int64),
                                ref["e_idx"][ir].astype(np.int64), tiny.t_start, tiny.t_end)
    e_in = np.abs(got["t_in"][ig] - ref["t_in"][ir])[well] / T[well]
    e_out = np.abs(got["t_out"][ig] - ref["t_out"][ir])[well] / T[well]
    assert e_in.max() <= 1e-11 and e_out.max() <= 1e-11, (e_in.max(), e_out.max())


@pytest.mark.parametrize("kind", ["temporal", "spatiotemporal"])
def test_query_clipped_by_the_request_start(tiny, kind):
    """A request start T_s inside query segments: the query record then holds its position at
    T_s (one rounding), and a pair whose entry starts later advances the query from there (a
    second rounding, where the plain definition has one). The match set must equal the oracle's,
    and on well-conditioned pairs of exactly that kind (query clipped at T_s, entry starting after
    T_s) the interval ends must still agree with the oracle's to 1e-11 of the overlap."""
    d, Ts, Te = 25.0, 37.3, 52.3  # ~23,000 hits, ~370 of them of the clipped kind
    q = tiny.queries
    ref = oracle.search(tiny.db, q, Ts, Te, d)
    got, _, _ = _run(tiny.db, q, kind, d, Ts, Te)
    parity.compare(got, ref, tiny.db, q, Ts, Te, d)
    kg = (got["q_idx"].astype(np.int64) << 32) | got["e_idx"].astype(np.int64)
    kr = (ref["q_idx"].astype(np.int64) << 32) | ref["e_idx"].astype(np.int64)
    common, ig, ir = np.intersect1d(kg, kr, return_indices=True)
    qi = ref["q_idx"][ir].astype(np.int64)
    ei = ref["e_idx"][ir].astype(np.int64)
    clipped = (q.t0[qi] < Ts) & (q.t1[qi] > Ts) & (tiny.db.t0[ei] > Ts)
    well = clipped & (np.abs(ref["s_min"][ir] - d) > 1e-6 * d)
    assert well.sum() > 200, well.sum()
    T = parity.overlap_duration(tiny.db, q, qi, ei, Ts, Te)
    e_in = np.abs(got["t_in"][ig] - ref["t_in"][ir])[well] / T[well]
    e_out = np.abs(got["t_out"][ig] - ref["t_out"][ir])[well] / T[well]
    assert e_in.max() <= 1e-11 and e_out.max() <= 1e-11, (e_in.max(), e_out.max())


def test_deterministic_order(tiny):
    idx = api.ts_build_index(tiny.db, kind="spatiotemporal")
    a = api.ts_search(idx, tiny.queries, 5.0, 0, 70).to_host()
    b = api.ts_search(idx, tiny.queries, 5.0, 0, 70).to_host()
    for k in a:
        assert np.array_equal(a[k], b[k])


def test_temporal_index_worked_example_on_gpu():
    with open(os.path.join(GOLDEN, "temporal_index_example.json")) as f:
        g = json.load(f)
    t = np.array(g["segments_t_start_t_end"])
    rows = [seg((0, 0, 0), a, (1, 1, 1), b) for a, b in t]
    idx = api.ts_build_index(segset(rows), kind="temporal", t_bins=g["m"])
    exp = g["expected"]
    np.testing.assert_array_equal(api.ts_index_export(idx, "perm"), np.arange(15))
    np.testing.assert_array_equal(api.ts_index_export(idx, "bin_start"), exp["bin_start"])
    np.testing.assert_array_equal(api.ts_index_export(idx, "bin_end"), exp["bin_end"])
    off = api.ts_index_export(idx, "bin_off")
    np.testing.assert_array_equal(off[:-1], exp["bin_first"])
    np.testing.assert_array_equal(off[1:] - 1, exp["bin_last"])


@pytest.mark.parametrize("m", [1, 7, 100, 997])
def test_temporal_index_matches_oracle(tiny, m):
    db = tiny.db
    idx = api.ts_build_index(db, kind="temporal", t_bins=m)
    ref = oracle.temporal_index(db.t0, db.t1, m)
    np.testing.assert_array_equal(api.ts_index_export(idx, "perm"), ref["perm"])
    np.testing.assert_array_equal(api.ts_index_export(idx, "bin_start"), ref["bin_start"])
    np.testing.assert_array_equal(api.ts_index_export(idx, "bin_end"), ref["bin_end"])
    np.testing.assert_array_equal(api.ts_index_export(idx, "bin_off"), ref["bin_off"])
    info = idx.info()
    assert info["t_min"] == ref["tmin"] and info["bin_width"] == ref["b"]


@pytest.mark.parametrize("v", [1, 5, 16])
def test_spatiotemporal_index_matches_oracle(tiny, v):
    db = tiny.db
    m = 50
    idx = api.ts_build_index(db, kind="spatiotemporal", t_bins=m, sub_bins=v)
    info = idx.info()
    tref = oracle.temporal_index(db.t0, db.t1, m)
    perm = tref["perm"]
    lo_cols = [np.minimum(db.x0, db.x1), np.minimum(db.y0, db.y1), np.minimum(db.z0, db.z1)]
    hi_cols = [np.maximum(db.x0, db.x1), np.maximum(db.y0, db.y1), np.maximum(db.z0, db.z1)]
    for dim in range(3):
        lo, w, ve = oracle.st_params(lo_cols[dim], hi_cols[dim], v)
        assert (info["sub_lo"][dim], info["sub_w"][dim], info["sub_bins"][dim]) == (lo, w, ve)
        ids, off = oracle.st_dim(lo_cols[dim][perm], hi_cols[dim][perm], tref["bin_of"], m, lo,
                                 w, ve)
        np.testing.assert_array_equal(api.ts_index_export(idx, "st_ids", dim), ids)
        np.testing.assert_array_equal(api.ts_index_export(idx, "st_off", dim), off)


@pytest.mark.parametrize("m,v,Ts,Te", [(200, 8, 0.0, 70.0), (1, 1, 0.0, 70.0),
                                        (3, 64, -10.0, 30.0), (2000, 8, 12.5, 12.75),
                                        (20000, 16, 0.0, 70.0), (137, 5, 55.0, 200.0)])
def test_schedules_match_oracle(tiny, m, v, Ts, Te):
    """The device schedule (bin ranges from bracketed searches, subbins from boundary tables)
    equals the oracle's for bin counts from 1 to 20,000 and clipped query intervals."""
    db, q = tiny.db, tiny.queries
    d = 5.0
    w0 = np.maximum(q.t0, Ts)
    w1 = np.minimum(q.t1, Te)
    tref = oracle.temporal_index(db.t0, db.t1, m)
    idx = api.ts_build_index(db, kind="temporal", t_bins=m)
    sel, lo, hi = api.ts_schedule(idx, q, d, Ts, Te)
    rlo, rhi = oracle.temporal_schedule(tref, w0, w1)
    np.testing.assert_array_equal(lo, rlo)
    np.testing.assert_array_equal(hi, rhi)
    assert np.all(sel == 3)
    # spatiotemporal
    idx = api.ts_build_index(db, kind="spatiotemporal", t_bins=m, sub_bins=v)
    info = idx.info()
    dims = []
    lo_cols = [np.minimum(db.x0, db.x1), np.minimum(db.y0, db.y1), np.minimum(db.z0, db.z1)]
    hi_cols = [np.maximum(db.x0, db.x1), np.maximum(db.y0, db.y1), np.maximum(db.z0, db.z1)]
    for dim in range(3):
        ids, off = oracle.st_dim(lo_cols[dim][tref["perm"]], hi_cols[dim][tref["perm"]],
                                 tref["bin_of"], m, info["sub_lo"][dim], info["sub_w"][dim],
                                 info["sub_bins"][dim])
        dims.append({"lo": info["sub_lo"][dim], "w": info["sub_w"][dim],
                     "v": info["sub_bins"][dim], "off": off})
    qmin = [np.minimum(q.x0, q.x1), np.minimum(q.y0, q.y1), np.minimum(q.z0, q.z1)]
    qmax = [np.maximum(q.x0, q.x1), np.maximum(q.y0, q.y1), np.maximum(q.z0, q.z1)]
    rsel, rlo, rhi = oracle.st_schedule(tref, dims, qmin, qmax, w0, w1, d)
    sel, lo, hi = api.ts_schedule(idx, q, d, Ts, Te)
    np.testing.assert_array_equal(sel, rsel)
    np.testing.assert_array_equal(lo, rlo)
    np.testing.assert_array_equal(hi, rhi)
    if (m, v, Ts, Te) == (200, 8, 0.0, 70.0):
        assert (rsel < 3).sum() > 100  # some queries served by subbins


def test_analytic_cases_on_gpu():
    # head-on (hit [7.5, 12.5]), parallel at 0.999 d (whole window), perpendicular tangent
    # (single instant 10), parallel at 1.001 d (no hit), touching windows (no hit)
    d = 5.0
    q = segset([seg((-10, 0, 0), 0, (10, 0, 0), 20)])
    e = segset([
        seg((10, 0, 0), 0, (-10, 0, 0), 20),
        seg((-10, 4.995, 0), 0, (10, 4.995, 0), 20),
        seg((0, 5, 0), 0, (0, 5, 0), 20),
        seg((-10, 5.005, 0), 0, (10, 5.005, 0), 20),
        seg((10, 0, 0), 20, (11, 0, 0), 21),
    ])
    for kind in ("brute", "temporal", "spatiotemporal", "spatial"):
        idx = api.ts_build_index(e, kind=kind)
        got = api.ts_search(idx, q, d, -1e9, 1e9).to_host(sort=True)
        assert got["e_idx"].tolist() == [0, 1, 2], kind
        np.testing.assert_allclose(got["t_in"], [7.5, 0.0, 10.0], atol=1e-12)
        np.testing.assert_allclose(got["t_out"], [12.5, 20.0, 10.0], atol=1e-12)


def test_edge_cases():
    rng = np.random.default_rng(3)
    from tests.cases import random_segments
    db = random_segments(rng, 300, box=5.0)
    q = random_segments(rng, 50, box=5.0)
    idx = api.ts_build_index(db, kind="spatiotemporal")
    # empty query set
    empty = Segments.from_matrix(np.zeros((0, 8)))
    r = api.ts_search(idx, empty, 1.0, 0, 10)
    assert r.count == 0 and r.stats["n_queries"] == 0
    # interval outside every query window
    r = api.ts_search(idx, q, 1.0, 100.0, 200.0)
    assert r.count == 0 and r.stats["n_qsegs"] == 0
    # degenerate interval (t_start == t_end): no positive overlap anywhere
    r = api.ts_search(idx, q, 1.0, 5.0, 5.0)
    assert r.count == 0
    # huge d: every pair with a positive-length window is a hit
    ref = oracle.search(db, q, -1e9, 1e9, 1e6)
    got = api.ts_search(idx, q, 1e6, -1e9, 1e9).to_host(sort=True)
    parity.compare(got, ref, db, q, -1e9, 1e9, 1e6)
    # single-entry database
    one = db.take([7])
    idx1 = api.ts_build_index(one, kind="temporal")
    ref = oracle.search(one, q, 0, 20, 3.0)
    got = api.ts_search(idx1, q, 3.0, 0, 20).to_host(sort=True)
    parity.compare(got, ref, one, q, 0, 20, 3.0)


def test_invalid_inputs_are_rejected():
    rng = np.random.default_rng(4)
    from tests.cases import random_segments
    db = random_segments(rng, 100)
    bad = db.as_matrix().copy()
    bad[5, 2] = np.nan
    with pytest.raises(api.TsError) as e:
        api.ts_build_index(Segments.from_matrix(bad), kind="temporal")
    assert e.value.status == 1
    bad = db.as_matrix().copy()
    bad[3, 7] = bad[3, 3]  # t_end == t_start
    with pytest.raises(api.TsError):
        api.ts_build_index(Segments.from_matrix(bad), kind="temporal")
    idx = api.ts_build_index(db, kind="temporal")
    for d in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(api.TsError):
            api.ts_search(idx, db, d, 0, 10)
    with pytest.raises(api.TsError):
        api.ts_search(idx, db, 1.0, 10, 0)
    qbad = db.as_matrix().copy()
    qbad[0, 0] = np.inf
    with pytest.raises(api.TsError):
        api.ts_search(idx, Segments.from_matrix(qbad), 1.0, 0, 10)


def test_result_capacity_reports_exact_count(tiny):
    idx = api.ts_build_index(tiny.db, kind="temporal")
    full = api.ts_search(idx, tiny.queries, 5.0, 0, 70)
    n = full.count
    capped = api.ts_search(idx, tiny.queries, 5.0, 0, 70, max_results=n - 1)
    assert capped.status == 4 and capped.count == n
    ok = api.ts_search(idx, tiny.queries, 5.0, 0, 70, max_results=n)
    assert ok.status == 0 and ok.count == n


def test_device_tensor_inputs(tiny):
    import torch
    cols = {f: torch.from_numpy(getattr(tiny.db, f)).cuda() for f in Segments.FIELDS}
    qcols = {f: torch.from_numpy(getattr(tiny.queries, f)).cuda() for f in Segments.FIELDS}
    idx = api.ts_build_index(cols, kind="spatiotemporal")
    got = api.ts_search(idx, qcols, 5.0, 0, 70).to_host(sort=True)
    ref = oracle.search(tiny.db, tiny.queries, 0, 70, 5.0)
    parity.compare(got, ref, tiny.db, tiny.queries, 0, 70, 5.0)


@pytest.mark.parametrize("g", [1, 5, 50])
def test_grid_index_and_schedule_match_oracle(tiny, g):
    db, q = tiny.db, tiny.queries
    d, Ts, Te = 5.0, 0.0, 70.0
    idx = api.ts_build_index(db, kind="spatial", grid_cells=g)
    info = idx.info()
    tref = oracle.temporal_index(db.t0, db.t1, 1)
    perm = tref["perm"]
    emin = [np.minimum(db.x0, db.x1), np.minimum(db.y0, db.y1), np.minimum(db.z0, db.z1)]
    emax = [np.maximum(db.x0, db.x1), np.maximum(db.y0, db.y1), np.maximum(db.z0, db.z1)]
    lo, w = zip(*[oracle.grid_params(emin[k], emax[k], g) for k in range(3)])
    assert tuple(info["grid_lo"]) == lo and tuple(info["grid_w"]) == w
    A, off = oracle.grid1([e[perm] for e in emin], g, lo, w)
    np.testing.assert_array_equal(api.ts_index_export(idx, "perm"), perm)
    np.testing.assert_array_equal(api.ts_index_export(idx, "grid_a"), A)
    np.testing.assert_array_equal(api.ts_index_export(idx, "grid_off"), off)
    longest = [float((emax[k] - emin[k]).max()) for k in range(3)]
    qmin = [np.minimum(q.x0, q.x1), np.minimum(q.y0, q.y1), np.minimum(q.z0, q.z1)]
    qmax = [np.maximum(q.x0, q.x1), np.maximum(q.y0, q.y1), np.maximum(q.z0, q.z1)]
    w0 = np.maximum(q.t0, Ts)
    w1 = np.minimum(q.t1, Te)
    runs, cand = oracle.grid1_candidates(g, lo, w, longest, off, qmin, qmax, w0, w1, d)
    sel, glo, ghi = api.ts_schedule(idx, q, d, Ts, Te)
    assert np.all(sel == 4)
    np.testing.assert_array_equal(glo, runs)
    np.testing.assert_array_equal(ghi, cand)
    res = api.ts_search(idx, q, d, Ts, Te)
    assert res.stats["n_tests"] == int(cand.sum())  # one cell per entry: no duplicate candidates


def test_measured_alu_peaks_are_plausible():
    """The roofline denominators measured on the device: FP32 FMA well above FP64 FMA, both
    within the range a GPU of this class can reach."""
    p = api.ts_measure_alu_peaks()
    assert 10.0 < p["fp32_tflops"] < 400.0
    assert 0.05 < p["fp64_tflops"] < p["fp32_tflops"]


@pytest.mark.parametrize("kind", ["temporal", "spatiotemporal", "spatial"])
def test_sweep_counters_are_consistent(tiny, kind):
    """The count pass's sweep counters: chunks swept bound the bitmask chunks, every candidate
    that reached the FP64 test passed the FP32 filters of a swept chunk, and the hits are among
    the FP64 tests."""
    w = tiny
    idx = api.ts_build_index(w.db, kind=kind)
    res = api.ts_search(idx, w.queries, 5.0, 0.0, 70.0)
    st = res.stats
    assert st["n_tests"] > 0 and st["n_chunks"] > 0
    assert st["n_dense"] <= st["n_chunks"]
    assert st["n_sparse"] <= 32 * st["n_chunks"]  # (at most one visit per member and chunk)
    assert st["n_hits"] <= st["n_exact"] <= st["n_tests"]
    res.free()
    idx.free()


def test_st_schedule_widens_an_expanded_extent_that_lands_on_a_boundary():
    """The same hand case as the oracle's pin: subbins of width 10 from 0 in every dimension
    (entries spanning [0, 40], four subbins); a query at y = z = 20 with d = 2 meets two subbins
    in y and in z. Query A (x in [12, 12.5]) has its d-expanded x extent start exactly at the
    boundary 10: the relative widening makes it meet [0,10) too, so the temporal range serves it
    (selector 3, all seven entries). Query B (x from 12.5) meets only [10,20): the x subbin serves
    it, one entry (x = 15)."""
    pts = [(0, 0, 0), (40, 40, 40), (5, 20, 20), (9.5, 20, 20), (15, 20, 20), (25, 20, 20),
           (35, 20, 20)]
    db = segset([seg(p, 0, p, 1) for p in pts])
    q = segset([seg((12, 20, 20), 0, (12.5, 20, 20), 1), seg((12.5, 20, 20), 0, (13, 20, 20), 1)])
    idx = api.ts_build_index(db, kind="spatiotemporal", t_bins=1, sub_bins=4)
    info = idx.info()
    assert list(info["sub_bins"]) == [4, 4, 4]
    assert list(info["sub_lo"]) == [0.0, 0.0, 0.0] and list(info["sub_w"]) == [10.0, 10.0, 10.0]
    sel, lo, hi = api.ts_schedule(idx, q, 2.0, 0.0, 1.0)
    assert sel[0] == 3 and hi[0] - lo[0] == 7
    assert sel[1] == 0 and hi[1] - lo[1] == 1
    got = api.ts_search(idx, q, 2.0, 0.0, 1.0).to_host(sort=True)
    ref = oracle.search(db, q, 0.0, 1.0, 2.0)
    parity.compare(got, ref, db, q, 0.0, 1.0, 2.0)
    idx.free()
