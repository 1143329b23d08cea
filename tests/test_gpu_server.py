"""Served search: requests from several threads through the request loop; each result must equal
the same request searched alone (plain ts_search), whatever batch it shared."""
import threading

import numpy as np
import pytest

from paper_1410_2698_gb300 import api, workloads
from paper_1410_2698_gb300.workloads import Segments

pytestmark = pytest.mark.gpu


def _stream(w, n, seed):
    rng = np.random.default_rng(seed)
    seg_per = w.queries.n // len(w.query_traj_ids)
    out = []
    for _ in range(n):
        k = int(rng.integers(1, 6))
        pick = rng.choice(len(w.query_traj_ids), size=k, replace=False)
        L = int(rng.integers(3, seg_per + 1))
        s0 = int(rng.integers(0, seg_per - L + 1))
        idx = (pick[:, None] * seg_per + s0 + np.arange(L)[None, :]).ravel()
        q = w.queries.take(idx)
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(10.0))))
        out.append((q, d, float(q.t0.min()), float(q.t1.max())))
    return out


def _same(a, b):
    for k in ("q_idx", "e_idx", "t_in", "t_out"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("kind,use_graph", [("spatiotemporal", True), ("temporal", False),
                                            ("spatial", True)])
def test_served_results_equal_alone(kind, use_graph):
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind=kind)
    reqs = _stream(w, 60, seed=11)
    srv = api.Server(idx, max_batch_requests=8, max_batch_queries=4000, max_batch_rows=200000,
                     max_inflight=2, use_graph=use_graph, linger_us=300)
    tickets = [None] * len(reqs)

    def client(lo, hi):
        for i in range(lo, hi):
            q, d, ts, te = reqs[i]
            tickets[i] = srv.submit(q, d, ts, te)

    ths = [threading.Thread(target=client, args=(a, a + 30)) for a in (0, 30)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    batch_sizes = []
    for i, req in enumerate(reqs):
        res, tm = srv.wait(tickets[i], timeout_ms=60000)
        assert tm["submit_us"] <= tm["start_us"] <= tm["done_us"]
        batch_sizes.append(tm["batch_requests"])
        q, d, ts, te = req
        alone = api.ts_search(idx, q, d, ts, te).to_host(sort=True)
        _same(res.to_host(sort=True), alone)
        res.free()
    srv.close()
    assert max(batch_sizes) > 1  # requests did share batches


def test_server_splits_overflowing_batches_and_rejects_oversized_requests():
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind="temporal")
    reqs = _stream(w, 12, seed=3)
    counts = [api.ts_search(idx, q, d, ts, te).count for q, d, ts, te in reqs]
    cap = max(counts) + 1  # every request fits alone, a batch of several usually does not
    srv = api.Server(idx, max_batch_requests=12, max_batch_queries=4000, max_batch_rows=cap,
                     max_inflight=1, linger_us=2000)
    tickets = [srv.submit(q, d, ts, te) for q, d, ts, te in reqs]
    for t, req, n in zip(tickets, reqs, counts):
        res, _ = srv.wait(t)
        assert res.count == n
        res.free()
    # a request with more rows than a batch holds ends with TS_ERR_CAPACITY
    small = api.Server(idx, max_batch_requests=4, max_batch_queries=4000, max_batch_rows=2)
    t = small.submit(w.queries, 5.0, 0.0, 70.0)
    with pytest.raises(api.TsError) as e:
        small.wait(t)
    assert e.value.status == 4
    small.close()
    srv.close()


def test_server_wait_is_bounded_and_cancel_works():
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind="temporal")
    srv = api.Server(idx, max_batch_requests=2, max_batch_queries=4000, max_batch_rows=400000,
                     max_inflight=1, linger_us=0)
    tickets = [srv.submit(w.queries, 5.0, 0.0, 70.0) for _ in range(6)]
    # the last request is very likely still queued behind five full searches
    try:
        srv.cancel(tickets[-1])
        cancelled = True
    except api.TsError as e:
        assert e.status == 1  # already started
        cancelled = False
    try:
        res, _ = srv.wait(tickets[0], timeout_ms=0)
        res.free()
    except api.TsError as e:
        assert e.status == 5  # not done yet: the wait ends at its limit
        res, _ = srv.wait(tickets[0], timeout_ms=60000)
        res.free()
    for t in tickets[1:-1]:
        srv.wait(t)[0].free()
    if cancelled:
        with pytest.raises(api.TsError) as e:
            srv.wait(tickets[-1])
        assert e.value.status == 6
    else:
        srv.wait(tickets[-1])[0].free()
    srv.close()
