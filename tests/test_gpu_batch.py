"""Batched search: many requests (own query sets, distances and intervals) in one pipeline, as a
one-shot call and as a reusable plan replayed as a CUDA graph. Every request's rows must equal
the plain single-request search, alone versus in the mix."""
import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads
from paper_1410_2698_gb300.workloads import Segments
from tests import parity

pytestmark = pytest.mark.gpu


def _requests(w, rng, n_req, max_traj=8):
    """Requests of whole query trajectories with their own d and interval; one request is empty
    and one has an interval before every query."""
    seg_per = w.queries.n // len(w.query_traj_ids)
    reqs = []
    for r in range(n_req):
        k = int(rng.integers(1, max_traj + 1))
        pick = rng.choice(len(w.query_traj_ids), size=k, replace=False)
        idx = (pick[:, None] * seg_per + np.arange(seg_per)[None, :]).ravel()
        q = w.queries.take(idx)
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(10.0))))
        ts = float(q.t0.min() + rng.uniform(0, 5))
        te = float(q.t1.max() - rng.uniform(0, 5))
        reqs.append((q, d, ts, max(ts, te)))
    reqs.append((Segments.from_matrix(np.zeros((0, 8))), 1.0, 0.0, 10.0))
    q0 = reqs[0][0]
    reqs.append((q0, 2.0, -100.0, -50.0))
    return reqs


def _plain(idx, req):
    q, d, ts, te = req
    return api.ts_search(idx, q, d, ts, te).to_host(sort=True)


def _same(a, b):
    for k in ("q_idx", "e_idx", "t_in", "t_out"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("kind", ["temporal", "spatiotemporal", "spatial", "brute"])
def test_one_shot_batch_equals_plain(kind):
    w = workloads.tiny()
    rng = np.random.default_rng(5)
    reqs = _requests(w, rng, 9)
    idx = api.ts_build_index(w.db, kind=kind)
    outs = api.ts_search_batch(idx, reqs)
    assert len(outs) == len(reqs)
    for req, res in zip(reqs, outs):
        _same(res.to_host(sort=True), _plain(idx, req))
    # a request's rows against the oracle as well
    q, d, ts, te = reqs[1]
    parity.compare(outs[1].to_host(sort=True), oracle.search(w.db, q, ts, te, d), w.db, q, ts,
                   te, d)


@pytest.mark.parametrize("use_graph", [False, True])
def test_plan_runs_equal_plain(use_graph):
    import torch
    w = workloads.tiny()
    rng = np.random.default_rng(9)
    idx = api.ts_build_index(w.db, kind="spatiotemporal")
    plan = api.BatchPlan(idx, max_requests=16, max_queries=4000, max_rows=400000,
                         use_graph=use_graph)
    pinned_out = {k: torch.empty(400000, dtype=dt, pin_memory=True).numpy()
                  for k, dt in (("q_idx", torch.int32), ("e_idx", torch.int32),
                                ("t_in", torch.float64), ("t_out", torch.float64))}
    for k in ("q_idx", "e_idx"):
        pinned_out[k] = pinned_out[k].view(np.uint32)
    for trial in range(4):
        reqs = _requests(w, rng, 6)
        if trial == 2:  # device-resident query columns
            reqs = [({f: torch.from_numpy(np.ascontiguousarray(getattr(q, f))).cuda()
                      for f in Segments.FIELDS} if q.n else q, d, ts, te)
                    for q, d, ts, te in reqs]
        if trial == 3:  # pinned host columns (read in place) mixed with pageable ones (staged)
            reqs = [({f: torch.from_numpy(np.ascontiguousarray(getattr(q, f))).pin_memory()
                      for f in Segments.FIELDS} if r % 2 == 0 and q.n else q, d, ts, te)
                    for r, (q, d, ts, te) in enumerate(reqs)]
        if trial == 1:  # marshalled once, run twice
            prepared = api.prepare_requests(reqs)
            plan.run(prepared)
            plan.wait()
            plan.run(prepared)
        else:
            plan.run(reqs)
        st = plan.wait()
        assert not st["overflow"] and st["nreq"] == len(reqs)
        total = 0
        for r, req in enumerate(reqs):
            if trial == 3:  # rows into preallocated pinned buffers
                got = {k: v.copy() for k, v in plan.request_to_host(r, out=pinned_out).items()}
                o = np.lexsort((got["e_idx"], got["q_idx"]))
                got = {k: v[o] for k, v in got.items()}
            else:
                got = plan.request_to_host(r, sort=True)
            q, d, ts, te = req
            qh = q if isinstance(q, Segments) else Segments(
                *[q[f].cpu().numpy() for f in Segments.FIELDS], traj=np.zeros(0, np.uint32))
            _same(got, _plain(idx, (qh, d, ts, te)))
            total += got["q_idx"].size
        assert total == st["rows"]
        # every row of the run in one copy: each request's span equals its own copy
        allrows, spans = plan.rows_to_host()
        assert len(spans) == len(reqs) and sum(n for _, n in spans) == st["rows"]
        for r, (f, n) in enumerate(spans):
            own = plan.request_to_host(r)
            for k in ("q_idx", "e_idx", "t_in", "t_out"):
                assert np.array_equal(allrows[k][f:f + n], own[k]), k
    plan.free()


def test_plans_sharing_a_stream_are_waited_for_one_by_one():
    """Plans run one after another on one stream (the end-to-end step's order for large plans):
    waiting for the first waits for its own run, its rows are read on its own stream while the
    second plan's run may still be on the shared stream, and every request of both plans equals
    its plain search."""
    import torch
    w = workloads.tiny()
    rng = np.random.default_rng(21)
    idx = {k: api.ts_build_index(w.db, kind=k) for k in ("temporal", "spatial")}
    plans = {k: api.BatchPlan(idx[k], max_requests=8, max_queries=4000, max_rows=400000,
                              use_graph=True) for k in idx}
    shared = torch.cuda.Stream()
    for trial in range(2):
        reqs = _requests(w, rng, 5)
        for k in plans:
            plans[k].run(reqs, stream=shared.cuda_stream)
        for k in plans:
            st = plans[k].wait()
            assert not st["overflow"] and st["nreq"] == len(reqs)
            rows, spans = plans[k].rows_to_host()
            assert sum(n for _, n in spans) == st["rows"]
            for r, req in enumerate(reqs):
                f, n = spans[r]
                got = {c: v[f:f + n] for c, v in rows.items()}
                o = np.lexsort((got["e_idx"], got["q_idx"]))
                _same({c: v[o] for c, v in got.items()}, _plain(idx[k], req))
    for k in plans:
        plans[k].free()
        idx[k].free()


@pytest.mark.parametrize("kind", ["temporal", "spatial"])
def test_plan_rows_equal_with_and_without_scratch(kind):
    """The count pass keeps its hits for placement after the scan; the tiles with hits that a
    too small scratch could not keep are swept again by the write pass. Every scratch size (all
    hits kept, one, a few, half, all but one) gives the same rows in the same order."""
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind=kind)
    reqs = [(w.queries, d, 0.0, 70.0) for d in (1.0, 5.0)]
    out = []
    sizes = [0]
    while sizes:
        scratch = sizes.pop(0)
        plan = api.BatchPlan(idx, max_requests=2, max_queries=4000, max_rows=400000,
                             max_units=1 << 20, use_graph=True, scratch_rows=scratch)
        plan.run(reqs)
        st = plan.wait()
        assert not st["overflow"]
        assert st["rows"] > 8
        out.append([plan.request_to_host(r) for r in range(len(reqs))])
        plan.free()
        if scratch == 0:
            n = st["rows"]
            sizes = [1, 8, n // 2, n - 1]
    for other in out[1:]:
        for a, b in zip(out[0], other):
            _same(a, b)  # unsorted: the same row order
    for r, req in enumerate(reqs):
        b = out[0][r]
        order = np.lexsort((b["e_idx"], b["q_idx"]))
        _same({k: v[order] for k, v in b.items()}, _plain(idx, req))


def test_plan_reports_overflow_with_exact_count():
    w = workloads.tiny()
    idx = api.ts_build_index(w.db, kind="temporal")
    plan = api.BatchPlan(idx, max_requests=2, max_queries=4000, max_rows=100, use_graph=True)
    plan.run([(w.queries, 5.0, 0.0, 70.0)])
    st = plan.wait()
    ref = api.ts_search(idx, w.queries, 5.0, 0.0, 70.0).count
    assert st["overflow"] and st["rows"] == ref
    # the next run within capacity succeeds on the same plan and graph
    small = w.queries.take(np.arange(3))
    plan.run([(small, 0.5, 0.0, 70.0)])
    st = plan.wait()
    assert not st["overflow"]
    _same(plan.request_to_host(0, sort=True), _plain(idx, (small, 0.5, 0.0, 70.0)))
