"""Autotuner for the batched search: bin granularity of the index (temporal bins m, subbins v,
grid cells g), records per work tile and pair-kernel blocks, chosen by timing a sample batch of
requests through the C ABI. Results are cached per (workload signature, GPU name) in a JSON file.

The tuner only measures; every candidate runs the same CUDA path (same results, checked by row
counts), so the choice affects speed only.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ts_gb300_autotune.json")

SPACE = {
    "temporal": {"t_bins": [0.25, 0.5, 1, 2, 4, 8]},     # multiples of span / longest duration
    "spatiotemporal": {"t_bins": [1, 4], "sub_bins": [4, 8, 16, 32, 64]},
    "spatial": {"grid_cells": [10, 25, 50, 100]},
}
TILES = [128, 256, 512, 1024, 2048]


def signature(db, requests, kind) -> str:
    """Stable key of a workload: database size and extent, request count and sizes, kind."""
    h = hashlib.sha256()
    h.update(kind.encode())
    h.update(np.array([db.n, len(requests)], dtype=np.int64).tobytes())
    for col in (db.x0, db.y0, db.z0, db.t0, db.t1):
        h.update(np.array([col.min(), col.max()], dtype=np.float64).tobytes())
    for q, d, ts, te in requests[:64]:
        h.update(np.array([q.n if hasattr(q, "n") else 0, d, ts, te], dtype=np.float64).tobytes())
    return h.hexdigest()[:24]


def sm_count() -> int:
    """Streaming multiprocessors of the current device (152 on a GB300)."""
    try:
        import torch
        return int(torch.cuda.get_device_properties(torch.cuda.current_device())
                   .multi_processor_count)
    except Exception:  # pragma: no cover
        return 152


def step_grids(sms=None):
    """Pair-kernel grids the overlapped step is tuned over: all resident blocks (0), then 1.75,
    1.5, 1.25 and 1 blocks per SM."""
    sms = sms or sm_count()
    return (0, (7 * sms) // 4, (3 * sms) // 2, (5 * sms) // 4, sms)


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:  # pragma: no cover
        return "unknown"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _units(index, requests, kind):
    """Unit capacity of a plan: grid indexes hold one unit per z-run of a query's cells (counted
    by the schedule); the other indexes one per query (0 = the plan's default)."""
    if kind != "spatial":
        return 0
    u = sum(int(api.ts_schedule(index, q, d, ts, te)[1].sum()) for q, d, ts, te in requests)
    return u + u // 10 + 1024


def _time_plan(index, requests, tile, pair_blocks, max_rows, repeats, units=0):
    """Best wall time of `repeats` runs of a plan over the requests (after a warm-up run that
    also captures the graph). A run that outgrows the plan's rows or tiles is retried with the
    exact counts the device reported."""
    tiles = 0
    st = None
    for _ in range(3):
        plan = api.BatchPlan(index, max_requests=len(requests),
                             max_queries=sum(q.n for q, *_ in requests), max_rows=max_rows,
                             tile_records=tile, use_graph=True, pair_blocks=pair_blocks,
                             max_units=units, max_tiles=tiles)
        try:
            plan.run(requests)
            st = plan.wait()  # warm-up (and graph capture)
            if st["overflow"]:
                max_rows = max(max_rows, st["rows"] + st["rows"] // 10 + 1024)
                tiles = max(tiles, 2 * st["stats"]["n_tiles"] + 65536)
                continue
            best = float("inf")
            for _ in range(repeats):
                t0 = time.perf_counter()
                plan.run(requests)
                st = plan.wait()
                best = min(best, time.perf_counter() - t0)
            return best, st
        finally:
            plan.free()
    return None, st


def tune(db, requests, kind, cache_path=DEFAULT_CACHE, repeats=3, max_rows=1 << 24,
         index_budget=6, force=False):
    """Return the best {index params, tile_records, pair_blocks} for `kind` on this workload.
    requests: list of (queries, d, t_start, t_end) used as the timing sample."""
    key = f"{signature(db, requests, kind)}|{_gpu_name()}"
    cache = _load(cache_path)
    if not force and key in cache:
        return cache[key]
    span = float(db.t1.max() - db.t0.min())
    longest = float((db.t1 - db.t0).max())
    base = max(1.0, span / max(longest, 1e-300))
    candidates = []
    space = SPACE.get(kind, {})
    if kind == "temporal":
        for f in space["t_bins"]:
            candidates.append({"t_bins": int(max(1, min(db.n, round(f * base))))})
    elif kind == "spatiotemporal":
        for f in space["t_bins"]:
            for v in space["sub_bins"]:
                candidates.append({"t_bins": int(max(1, min(db.n, round(f * base)))),
                                   "sub_bins": v})
    elif kind == "spatial":
        candidates = [{"grid_cells": g} for g in space["grid_cells"]]
    else:
        candidates = [{}]
    candidates = candidates[:max(index_budget, 1)] if len(candidates) > index_budget else candidates
    trials = []
    best = None
    rows = None
    for params in candidates:
        idx = api.ts_build_index(db, kind=kind, **params)
        try:
            t, st = _time_plan(idx, requests, 256, 0, max_rows, repeats,
                               _units(idx, requests, kind))
        finally:
            idx.free()
        if t is None:
            continue
        if rows is None:
            rows = st["rows"]
        if st["rows"] != rows:
            raise RuntimeError("autotune: candidates disagree on the result count")
        trials.append({"params": params, "s": t})
        if best is None or t < best[1]:
            best = (params, t)
    if best is None:
        raise RuntimeError("autotune: every candidate overflowed max_rows")
    idx = api.ts_build_index(db, kind=kind, **best[0])
    tile_best = (256, 0, best[1])
    units = _units(idx, requests, kind)
    try:
        for tile in TILES:
            for pb in (0, sm_count()):  # all resident blocks, or one block per SM
                t, st = _time_plan(idx, requests, tile, pb, max_rows, repeats, units)
                if t is not None:
                    trials.append({"params": dict(best[0]), "tile_records": tile,
                                   "pair_blocks": pb, "s": t})
                    if t < tile_best[2]:
                        tile_best = (tile, pb, t)
    finally:
        idx.free()
    out = {"index": best[0], "tile_records": tile_best[0], "pair_blocks": tile_best[1],
           "seconds": tile_best[2], "trials": trials, "rows": rows}
    cache[key] = out
    _store(cache_path, cache)
    return out


STUDY = {
    "temporal": ("t_bins", [0.25, 0.5, 1, 2, 4, 8, 16]),     # multiples of span / longest duration
    "spatiotemporal": ("sub_bins", [1, 2, 4, 8, 16, 32, 64]),
    "spatial": ("grid_cells", [5, 10, 25, 50, 100, 200]),
}


def time_overlapped(plans, requests, order, warmup=8, reps=20):
    """Wall time of `reps` steps that launch every plan (each on its own stream) in `order`, then
    wait for each; `warmup` untimed steps first (the first also captures the plans' graphs)."""
    for _ in range(warmup):
        for k in order:
            plans[k].run(requests, stream=0)
        for k in order:
            plans[k].wait()
    t0 = time.perf_counter()
    for _ in range(reps):
        for k in order:
            plans[k].run(requests, stream=0)
        for k in order:
            plans[k].wait()
    return time.perf_counter() - t0


def tune_overlapped(make_plans, kinds, requests, grids=None, tune_grid=True,
                    timer=time_overlapped):
    """Tune a step that runs several plans at once (one per kind, overlapping on their streams):
    first the persistent pair kernel's grid shared by the plans (`grids`, 0 = all resident
    blocks; a pair kernel holds the SMs it runs on, so a smaller grid leaves room for the other
    plans' kernels), then the order in which the plans are launched. make_plans(pair_blocks)
    returns {kind: plan}; the plans it returns are freed here. Returns (pair_blocks, order)."""
    import itertools
    grids = step_grids() if grids is None else grids
    pair_blocks = None
    if tune_grid:
        best = None
        for pb in grids:
            plans = make_plans(pb)
            try:
                dt = timer(plans, requests, list(kinds))
            finally:
                for pl in plans.values():
                    pl.free()
            if best is None or dt < best[1]:
                best = (pb, dt)
        pair_blocks = best[0]
    plans = make_plans(pair_blocks)
    try:
        best = None
        for seq in itertools.permutations(kinds):
            dt = timer(plans, requests, list(seq))
            if best is None or dt < best[1]:
                best = (list(seq), dt)
    finally:
        for pl in plans.values():
            pl.free()
    return pair_blocks, best[0]


def study(db, queries, distances, t_start, t_end, kinds=("temporal", "spatiotemporal", "spatial"),
          repeats=3):
    """Response of the search to the index's bin granularity (the temporal bins m, the subbins v,
    the grid cells g) at every distance: one record per (kind, value, d) with the plain search's
    wall time (median of `repeats`), its count-pass time, the candidate tests, FP64 tests and hits,
    and for subbins the fraction of query segments served by a subbin."""
    span = float(db.t1.max() - db.t0.min())
    longest = float((db.t1 - db.t0).max())
    base = max(1.0, span / max(longest, 1e-300))
    out = []
    for kind in kinds:
        name, values = STUDY[kind]
        for v in values:
            param = int(max(1, min(db.n, round(v * base)))) if name == "t_bins" else int(v)
            idx = api.ts_build_index(db, kind=kind, **{name: param})
            try:
                for d in distances:
                    times = []
                    st = None
                    for _ in range(repeats + 1):
                        t0 = time.perf_counter()
                        r = api.ts_search(idx, queries, d, t_start, t_end)
                        times.append(time.perf_counter() - t0)
                        st = r.stats
                        r.free()
                    times = sorted(times[1:])
                    nq = max(st["n_qsegs"], 1)
                    out.append({"kind": kind, name: param, "d": d,
                                "ms": 1e3 * times[len(times) // 2],
                                "count_pass_ms": st["ms_count_pass"], "tests": st["n_tests"],
                                "exact": st["n_exact"], "hits": st["n_hits"],
                                "subbin_fraction": st["n_subbin"] / nq
                                if kind == "spatiotemporal" else None})
            finally:
                idx.free()
    return out
