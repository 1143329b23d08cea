"""The all-pairs search that allocates nothing (ts_search_brute_noalloc).

It serves callers that cannot allocate device memory themselves through the library, e.g. code
inside an application that owns all device memory through its own allocator, or latency-bound
request paths that cannot afford cudaMalloc. The test calls it through the C ABI twice in a row
(it reuses one fixed scratch array between calls) and checks each result against the indexed
search entry point (ts_search on a brute-force index), within the tolerance of the other GPU
parity tests. This file is collected last so a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_1410_2698_gb300 import api, workloads
from paper_1410_2698_gb300.workloads import Segments
from tests import parity

pytestmark = pytest.mark.gpu


def _dev(segs, torch):
    return {f: torch.from_numpy(np.ascontiguousarray(getattr(segs, f))).cuda()
            for f in Segments.FIELDS}


def test_noalloc_search_matches_ts_search_on_two_calls():
    import torch
    w = workloads.tiny()
    db, q = w.db, w.queries
    d, Ts, Te = w.distances[0], w.t_start, w.t_end
    idx = api.ts_build_index(db, kind="brute")
    ref = api.ts_search(idx, q, d, Ts, Te).to_host(sort=True)
    idx.free()
    assert ref["q_idx"].size > 1000
    dbd, qd = _dev(db, torch), _dev(q, torch)
    cap = ref["q_idx"].size + 64
    outs = []
    for _ in range(2):
        qi = torch.full((cap,), 0xFFFF, dtype=torch.int32, device="cuda")
        ei = torch.full((cap,), 0xFFFF, dtype=torch.int32, device="cuda")
        tin = torch.full((cap,), float("nan"), dtype=torch.float64, device="cuda")
        tout = torch.full((cap,), float("nan"), dtype=torch.float64, device="cuda")
        st, n = api.ts_search_brute_noalloc(dbd, qd, d, Ts, Te, qi, ei, tin, tout)
        torch.cuda.synchronize()
        assert st == 0 and n == ref["q_idx"].size
        got = {"q_idx": qi[:n].cpu().numpy().astype(np.uint32),
               "e_idx": ei[:n].cpu().numpy().astype(np.uint32),
               "t_in": tin[:n].cpu().numpy(), "t_out": tout[:n].cpu().numpy()}
        order = np.lexsort((got["e_idx"], got["q_idx"]))
        got = {k: v[order] for k, v in got.items()}
        parity.compare(got, ref, db, q, Ts, Te, d)
        outs.append(got)
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k])


def test_noalloc_search_reports_capacity_and_size_limits():
    import torch
    w = workloads.tiny()
    db = w.db.take(np.arange(3000))
    q = w.queries.take(np.arange(300))
    dbd, qd = _dev(db, torch), _dev(q, torch)
    one = [torch.empty((1,), dtype=t, device="cuda")
           for t in (torch.int32, torch.int32, torch.float64, torch.float64)]
    st, n = api.ts_search_brute_noalloc(dbd, qd, w.distances[0], w.t_start, w.t_end, *one)
    assert st == 4 and n > 1  # more rows than the one-row capacity; none written
    # a problem above the fixed tile limit is rejected before any device work: 2^31 database
    # segments (the columns are never read) x 300 query segments
    from paper_1410_2698_gb300 import _lib
    import ctypes
    lib = _lib.load()
    s_db, keep1 = api.make_segments(dbd)
    s_q, keep2 = api.make_segments(qd)
    s_db.n = 1 << 31
    qp = _lib.ts_query_params(1.0, 0.0, 70.0, 0)
    count = ctypes.c_uint64(0)
    st = lib.ts_search_brute_noalloc(ctypes.byref(s_db), ctypes.byref(s_q), ctypes.byref(qp),
                                     None, None, None, None, 0, ctypes.byref(count), None)
    assert st == 4
    assert "scratch limit" in lib.ts_last_error().decode()
