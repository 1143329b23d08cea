"""GPU parity at the benchmark workloads' sizes: the Random-walk 1M configuration in full (the
oracle's temporal pruning finishes it in seconds), and the dense and merger-like configurations
on seeded samples of query trajectories."""
import numpy as np
import pytest

import oracle
from paper_1410_2698_gb300 import api, workloads
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rw1m():
    return workloads.random_walk_1m()


@pytest.fixture(scope="module")
def rw1m_indexes(rw1m):
    out = {k: api.ts_build_index(rw1m.db, kind=k)
           for k in ("temporal", "spatiotemporal", "spatial")}
    yield out
    for idx in out.values():
        idx.free()


_RW1M_REF = {}


def _rw1m_ref(w, d):
    if d not in _RW1M_REF:
        _RW1M_REF[d] = oracle.search(w.db, w.queries, w.t_start, w.t_end, d)
    return _RW1M_REF[d]


@pytest.mark.parametrize("d", [1.0, 5.0, 10.0, 25.0])
def test_random_walk_1m_full(rw1m, rw1m_indexes, d):
    ref = _rw1m_ref(rw1m, d)
    counts = {}
    for kind, idx in rw1m_indexes.items():
        got = api.ts_search(idx, rw1m.queries, d, rw1m.t_start, rw1m.t_end).to_host(sort=True)
        parity.compare(got, ref, rw1m.db, rw1m.queries, rw1m.t_start, rw1m.t_end, d)
        counts[kind] = got["q_idx"].size
    # every query segment meets its own database twin over its whole extent
    assert ref["q_idx"].size >= rw1m.queries.n


@pytest.mark.parametrize("kind,params,tile", [
    ("temporal", {"t_bins": 250}, 1024),
    ("spatiotemporal", {"t_bins": 500, "sub_bins": 32}, 512),
    ("spatial", {"grid_cells": 25}, 256),
])
def test_random_walk_1m_batched_as_benchmarked(rw1m, kind, params, tile):
    """The benchmark's launch configuration: one plan per index with the four distances as its
    requests, replayed as a CUDA graph on its own stream with a 228-block pair grid, index
    parameters and tiles as the autotuner picks them on this workload; every request's rows
    against the oracle, on the second replay."""
    import torch
    from paper_1410_2698_gb300.workloads import Segments
    w = rw1m
    qdev = {f: torch.from_numpy(getattr(w.queries, f)).cuda() for f in Segments.FIELDS}
    reqs = [(qdev, d, w.t_start, w.t_end) for d in w.distances]
    idx = api.ts_build_index(w.db, kind=kind, **params)
    units = 0
    if kind == "spatial":
        units = sum(int(api.ts_schedule(idx, w.queries, d, w.t_start, w.t_end)[1].sum())
                    for d in w.distances)
        units += units // 10 + 1024
    plan = api.BatchPlan(idx, max_requests=len(reqs), max_queries=w.queries.n * len(reqs),
                         max_rows=1 << 20, use_graph=True, stream=0, tile_records=tile,
                         pair_blocks=228, max_units=units, max_tiles=1 << 20)
    try:
        for _ in range(2):
            plan.run(reqs, stream=0)
            st = plan.wait()
            assert not st["overflow"]
        for r, d in enumerate(w.distances):
            got = plan.request_to_host(r, sort=True)
            parity.compare(got, _rw1m_ref(w, d), w.db, w.queries, w.t_start, w.t_end, d)
    finally:
        plan.free()
        idx.free()


def _trajectory_sample(w, n_traj, seed):
    seg_per = w.queries.n // len(w.query_traj_ids)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(w.query_traj_ids), size=n_traj, replace=False))
    idx = (pick[:, None] * seg_per + np.arange(seg_per)[None, :]).ravel()
    return w.queries.take(idx)


@pytest.fixture(scope="module")
def dense_small():
    # the dense configuration's density (20,000 trajectories x 101 samples in [0,50]^3)
    return workloads.dense()


@pytest.fixture(scope="module")
def dense_indexes(dense_small):
    out = {k: api.ts_build_index(dense_small.db, kind=k)
           for k in ("temporal", "spatiotemporal", "spatial")}
    yield out
    for idx in out.values():
        idx.free()


@pytest.mark.parametrize("d", [0.5, 2.0])
def test_dense_full(dense_small, dense_indexes, d):
    """The dense configuration in full: all 500 query trajectories against the 2M segments."""
    w = dense_small
    ref = oracle.search(w.db, w.queries, w.t_start, w.t_end, d)
    for kind, idx in dense_indexes.items():
        got = api.ts_search(idx, w.queries, d, w.t_start, w.t_end).to_host(sort=True)
        parity.compare(got, ref, w.db, w.queries, w.t_start, w.t_end, d)
    assert ref["q_idx"].size > w.queries.n  # dense: more than the self matches


@pytest.fixture(scope="module")
def merger():
    return workloads.merger_like()


@pytest.fixture(scope="module")
def merger_indexes(merger):
    out = {k: api.ts_build_index(merger.db, kind=k)
           for k in ("temporal", "spatiotemporal", "spatial")}
    yield out
    for idx in out.values():
        idx.free()


@pytest.mark.parametrize("d", [1.0, 5.0])
def test_merger_like_sampled(merger, merger_indexes, d):
    """The merger-like configuration (20M segments) on a seeded 1% of its query trajectories
    (20 of 2,000), plain searches with every index and a batch plan against the oracle."""
    w = merger
    q = _trajectory_sample(w, 20, seed=11)
    ref = oracle.search(w.db, q, w.t_start, w.t_end, d)
    first = None
    for kind, idx in merger_indexes.items():
        got = api.ts_search(idx, q, d, w.t_start, w.t_end).to_host(sort=True)
        if first is None:
            parity.compare(got, ref, w.db, q, w.t_start, w.t_end, d)
            first = got
        else:  # every index returns the same rows (bit for bit, sorted)
            for key in ("q_idx", "e_idx", "t_in", "t_out"):
                assert np.array_equal(got[key], first[key]), (kind, key)
    plan = api.BatchPlan(merger_indexes["spatiotemporal"], max_requests=2, max_queries=2 * q.n,
                         max_rows=2 * ref["q_idx"].size + (1 << 16), max_tiles=1 << 22)
    half = q.take(np.arange(q.n // 2))
    plan.run([(q, d, w.t_start, w.t_end), (half, d, w.t_start, w.t_end)])
    st = plan.wait()
    assert not st["overflow"]
    batched = plan.request_to_host(0, sort=True)
    for key in ("q_idx", "e_idx", "t_in", "t_out"):
        assert np.array_equal(batched[key], first[key]), key
    plan.free()
    assert ref["q_idx"].size > 10 * q.n  # hit-dense: many neighbours per query segment


def test_served_on_merger_like_equals_alone(merger, merger_indexes):
    """Served requests on the resident merger-like database (small runs of core trajectories,
    own intervals and d) equal the same requests searched alone, and the oracle's rows."""
    w = merger
    rng = np.random.default_rng(23)
    seg_per = w.queries.n // len(w.query_traj_ids)
    reqs = []
    for _ in range(12):
        k = int(rng.integers(1, 4))
        pick = rng.choice(len(w.query_traj_ids), size=k, replace=False)
        L = int(rng.integers(10, 40))
        s0 = int(rng.integers(0, seg_per - L))
        idx = (pick[:, None] * seg_per + s0 + np.arange(L)[None, :]).ravel()
        q = w.queries.take(idx)
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(10.0))))
        reqs.append((q, d, float(q.t0.min()), float(q.t1.max())))
    index = merger_indexes["spatiotemporal"]
    srv = api.Server(index, max_batch_requests=8, max_batch_queries=1 << 16,
                     max_batch_rows=1 << 26, linger_us=500)
    tickets = [srv.submit(q, d, ts, te) for q, d, ts, te in reqs]
    for t, (q, d, ts, te) in zip(tickets, reqs):
        res, tm = srv.wait(t, timeout_ms=120000)
        got = res.to_host(sort=True)
        alone = api.ts_search(index, q, d, ts, te).to_host(sort=True)
        for key in ("q_idx", "e_idx", "t_in", "t_out"):
            assert np.array_equal(got[key], alone[key]), key
        parity.compare(got, oracle.search(w.db, q, ts, te, d), w.db, q, ts, te, d)
        res.free()
    srv.close()


def test_served_stream_shaped_requests_on_merger_like_match_the_oracle(merger, merger_indexes):
    """Requests shaped like the served stream (the stream generator itself: 1-5,000 query
    trajectories, log-uniform, each a random database trajectory cut to a run of 10-200
    segments; the runs' span as interval; d log-uniform in [0.5, 10]) through two servers on the
    resident merger-like database, every result against the oracle. The generator's first
    requests are kept while their query segments total at most 30,000 (larger ones are skipped,
    so the oracle stays within a minute). One server's row limit is one more than the largest
    request's rows, so batches of several requests are split; the other (temporal index, small
    tiles) starts with plans whose tile capacity the requests outgrow, so its plans grow. Each
    mechanism must have re-queued some batch."""
    w = merger
    stream = workloads.served_stream(w, n_requests=60, rate_per_s=1.0, seed_offset=5,
                                     max_traj=5000)
    reqs, total = [], 0
    for r in stream:
        if total + r.queries.n <= 30000:
            reqs.append(r)
            total += r.queries.n
    assert len(reqs) >= 8 and max(r.queries.n for r in reqs) >= 2000
    st_index = merger_indexes["spatiotemporal"]
    rows = [api.ts_search(st_index, r.queries, r.d, r.t_start, r.t_end).count for r in reqs]
    refs = [oracle.search(w.db, r.queries, r.t_start, r.t_end, r.d) for r in reqs]
    servers = [
        ("split", api.Server(st_index, max_batch_requests=8, max_batch_queries=1 << 17,
                             max_batch_rows=max(rows) + 1, max_inflight=2, linger_us=2000)),
        ("grow", api.Server(merger_indexes["temporal"], max_batch_requests=8,
                            max_batch_queries=1 << 15, max_batch_rows=1 << 30, max_inflight=2,
                            tile_records=64, linger_us=2000)),
    ]
    for name, srv in servers:
        tickets = [srv.submit(r.queries, r.d, r.t_start, r.t_end) for r in reqs]
        requeued = 0
        for t, r, n, ref in zip(tickets, reqs, rows, refs):
            res, tm = srv.wait(t, timeout_ms=300000)
            requeued += tm["requeued"]
            assert res.count == n
            got = res.to_host(sort=True)
            parity.compare(got, ref, w.db, r.queries, r.t_start, r.t_end, r.d)
            res.free()
        srv.close()
        assert requeued > 0, name
