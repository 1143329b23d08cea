"""Edge cases of the search against the oracle: ragged tiles, duplicate entries and tied start
times, coordinates far from the origin (the FP32 filters' outward rounding), and the largest bin,
subbin and grid parameters."""
import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads
from paper_1410_2698_gb300.workloads import Segments
from tests import parity
from tests.cases import random_segments

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile", [64, 192, 2048])
@pytest.mark.parametrize("kind", ["temporal", "spatiotemporal", "spatial"])
def test_ragged_tiles_equal_plain(kind, tile):
    """Tiles of one chunk, of three chunks and of the largest size: the batched rows equal the
    plain search's, whatever the tail of every merged range."""
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind=kind)
    reqs = [(w.queries, d, 3.0, 61.0) for d in (0.7, 4.0)]
    plan = api.BatchPlan(idx, max_requests=2, max_queries=4000, max_rows=400000,
                         max_units=1 << 20, tile_records=tile)
    plan.run(reqs)
    st = plan.wait()
    assert not st["overflow"]
    for r, (q, d, ts, te) in enumerate(reqs):
        got = plan.request_to_host(r, sort=True)
        ref = api.ts_search(idx, q, d, ts, te).to_host(sort=True)
        for k in ("q_idx", "e_idx", "t_in", "t_out"):
            assert np.array_equal(got[k], ref[k]), k
    plan.free()


def test_duplicates_and_tied_start_times():
    """A database with every segment twice and many equal start times: each copy is its own
    entry (reported once each), and the order of tied entries does not change the rows."""
    rng = np.random.default_rng(21)
    base = random_segments(rng, 400, box=20.0, t_range=(0, 10))
    m = base.as_matrix()
    m[:, 3] = np.round(m[:, 3])  # start times on a few integer instants
    m[:, 7] = m[:, 3] + rng.uniform(0.5, 2.0, m.shape[0])
    db = Segments.from_matrix(np.concatenate([m, m]))
    q = Segments.from_matrix(m[::7].copy())
    ref = oracle.search(db, q, 0.0, 12.0, 2.5)
    for kind in ("temporal", "spatiotemporal", "spatial", "brute"):
        idx = api.ts_build_index(db, kind=kind)
        got = api.ts_search(idx, q, 2.5, 0.0, 12.0).to_host(sort=True)
        parity.compare(got, ref, db, q, 0.0, 12.0, 2.5)
    # every hit appears for both copies of its entry
    e = ref["e_idx"] % base.n
    assert np.all(np.bincount(e, minlength=base.n)[np.unique(e)] % 2 == 0)


@pytest.mark.parametrize("offset", [1e4, 1e6])
def test_far_from_origin(offset):
    """All coordinates shifted far from the origin, where an FP32 box is coarse: the outward
    rounded filters still keep every pair the FP64 test accepts."""
    rng = np.random.default_rng(31)
    db = random_segments(rng, 600, box=10.0, t_range=(0, 20))
    q = random_segments(rng, 80, box=10.0, t_range=(0, 20))
    for s in (db, q):
        for f in ("x0", "x1", "y0", "y1"):
            setattr(s, f, getattr(s, f) + offset)
    ref = oracle.search(db, q, 0.0, 20.0, 2.0)
    assert ref["q_idx"].size > 100
    for kind in ("temporal", "spatiotemporal", "spatial"):
        idx = api.ts_build_index(db, kind=kind)
        got = api.ts_search(idx, q, 2.0, 0.0, 20.0).to_host(sort=True)
        parity.compare(got, ref, db, q, 0.0, 20.0, 2.0)


def test_largest_parameters():
    """One bin per entry, 4,096 subbins per dimension, 512 grid cells per dimension."""
    w = workloads.tiny()
    q = w.queries.take(np.arange(400))
    ref = oracle.search(w.db, q, 0.0, 70.0, 3.0)
    for kind, prm in (("temporal", {"t_bins": w.db.n}),
                      ("spatiotemporal", {"t_bins": 2000, "sub_bins": 4096}),
                      ("spatial", {"grid_cells": 512})):
        idx = api.ts_build_index(w.db, kind=kind, **prm)
        got = api.ts_search(idx, q, 3.0, 0.0, 70.0).to_host(sort=True)
        parity.compare(got, ref, w.db, q, 0.0, 70.0, 3.0)
