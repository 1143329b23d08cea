"""Stationary-point search (fixed positions over an interval): equal to the oracle's search of the
same points written as zero-length query segments, from host and from device coordinates."""
import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads
from paper_1410_2698_gb300.workloads import Segments
from tests import parity

pytestmark = pytest.mark.gpu


def _points_as_segments(x, y, z, ts, te):
    n = x.size
    return Segments(x, y, z, np.full(n, ts), x.copy(), y.copy(), z.copy(), np.full(n, te),
                    traj=np.zeros(n, np.uint32))


@pytest.mark.parametrize("kind", ["temporal", "spatiotemporal", "spatial", "brute"])
def test_points_equal_oracle(kind):
    import torch
    w = workloads.tiny()
    rng = np.random.default_rng(3)
    n = 300
    x, y, z = (rng.uniform(-10, 110, n) for _ in range(3))
    ts, te, d = 10.0, 40.0, 6.0
    q = _points_as_segments(x, y, z, ts, te)
    ref = oracle.search(w.db, q, ts, te, d)
    assert ref["q_idx"].size > 50
    idx = api.ts_build_index(w.db, kind=kind)
    got = api.ts_search_points(idx, x, y, z, d, ts, te).to_host(sort=True)
    parity.compare(got, ref, w.db, q, ts, te, d)
    dev = [torch.from_numpy(a).cuda() for a in (x, y, z)]
    got_d = api.ts_search_points(idx, *dev, d, ts, te).to_host(sort=True)
    for k in ("q_idx", "e_idx", "t_in", "t_out"):
        assert np.array_equal(got_d[k], got[k]), k


def test_points_reject_an_empty_interval():
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind="temporal")
    x = np.zeros(3)
    with pytest.raises(api.TsError):
        api.ts_search_points(idx, x, x, x, 1.0, 5.0, 5.0)
    empty = api.ts_search_points(idx, np.zeros(0), np.zeros(0), np.zeros(0), 1.0, 0.0, 5.0)
    assert empty.count == 0
