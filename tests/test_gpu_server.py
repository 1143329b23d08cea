"""Served search: requests from several threads through the request loop; each result must equal
the same request searched alone (plain ts_search), whatever batch it shared, and the oracle's
result for that request under the acceptance rule."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads
from paper_1410_2698_gb300.workloads import Segments
from tests import parity

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
        got = res.to_host(sort=True)
        alone = api.ts_search(idx, q, d, ts, te).to_host(sort=True)
        _same(got, alone)
        parity.compare(got, oracle.search(w.db, q, ts, te, d), w.db, q, ts, te, d)
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


def test_server_defers_a_batch_until_results_release_memory():
    """Admission by memory: with a budget that holds the plans and one request's rows but not
    two, a second request waits (its wait times out, the request is not failed) while the first
    result is held, and completes -- equal to the oracle -- once that result is released."""
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind="temporal")
    reqs = [(w.queries, 25.0, 0.0, 70.0), (w.queries.take(np.arange(1500)), 20.0, 0.0, 70.0)]
    rows = [api.ts_search(idx, q, d, ts, te).count for q, d, ts, te in reqs]
    kw = dict(max_batch_requests=1, max_batch_queries=4000, max_batch_rows=1 << 26,
              max_inflight=1, linger_us=0, scratch_rows=1 << 16, admit_wait_ms=60000)
    probe = api.Server(idx, mem_budget_bytes=1 << 40, **kw)
    plan_bytes = probe.info()["plan_bytes"]
    probe.close()
    assert plan_bytes > 0
    budget = plan_bytes + 24 * max(rows) + 24 * min(rows) // 2  # one request's rows, not two
    srv = api.Server(idx, mem_budget_bytes=budget, **kw)
    assert srv.info()["budget_bytes"] == budget
    t0 = srv.submit(*reqs[0])
    res0, tm0 = srv.wait(t0, timeout_ms=60000)
    assert res0.count == rows[0]
    assert srv.info()["held_bytes"] == 24 * rows[0]
    t1 = srv.submit(*reqs[1])
    with pytest.raises(api.TsError) as e:  # deferred: the budget is held by the first result
        srv.wait(t1, timeout_ms=1500)
    assert e.value.status == 5
    res0.free()
    res1, tm1 = srv.wait(t1, timeout_ms=60000)
    q, d, ts, te = reqs[1]
    got = res1.to_host(sort=True)
    parity.compare(got, oracle.search(w.db, q, ts, te, d), w.db, q, ts, te, d)
    assert tm1["done_us"] - tm1["submit_us"] >= 1.0e6  # it waited for the release
    res1.free()
    assert srv.info()["held_bytes"] == 0
    srv.close()


def test_server_admits_beyond_the_budget_after_the_admission_wait():
    """The budget is soft: a client that holds one result and waits on the next must not wait
    forever. With a budget that fits one request's rows and a 200 ms admission wait, the second
    request completes -- equal to the oracle -- while the first result is still held, and
    destroying a server whose batch waits for memory cancels that batch instead of hanging."""
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind="temporal")
    reqs = [(w.queries, 25.0, 0.0, 70.0), (w.queries.take(np.arange(1500)), 20.0, 0.0, 70.0)]
    rows = [api.ts_search(idx, q, d, ts, te).count for q, d, ts, te in reqs]
    kw = dict(max_batch_requests=1, max_batch_queries=4000, max_batch_rows=1 << 26,
              max_inflight=1, linger_us=0, scratch_rows=1 << 16)
    probe = api.Server(idx, mem_budget_bytes=1 << 40, **kw)
    plan_bytes = probe.info()["plan_bytes"]
    probe.close()
    budget = plan_bytes + 24 * max(rows) + 24 * min(rows) // 2
    srv = api.Server(idx, mem_budget_bytes=budget, admit_wait_ms=200, **kw)
    res0, _ = srv.wait(srv.submit(*reqs[0]), timeout_ms=60000)
    t1 = srv.submit(*reqs[1])
    res1, tm1 = srv.wait(t1, timeout_ms=60000)  # res0 still held
    assert tm1["done_us"] - tm1["submit_us"] >= 0.2e6
    assert srv.info()["held_bytes"] == 24 * (rows[0] + rows[1])
    q, d, ts, te = reqs[1]
    parity.compare(res1.to_host(sort=True), oracle.search(w.db, q, ts, te, d), w.db, q, ts,
                   te, d)
    res1.free()
    # a batch left waiting for memory when the server is destroyed is cancelled
    srv2 = api.Server(idx, mem_budget_bytes=budget, admit_wait_ms=60000, **kw)
    srv2.submit(*reqs[1])
    time.sleep(0.5)
    t0 = time.perf_counter()
    srv2.close()
    assert time.perf_counter() - t0 < 10.0
    res0.free()
    srv.close()
