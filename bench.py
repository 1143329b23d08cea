"""Benchmark of the GB300 trajectory distance threshold search.

Workload (default): the merger-like configuration -- two Plummer spheres of 50,000 particles
each, 201 samples (20,000,000 database segments, 1.28 GB of FP64 segments), 2,000 query
trajectories from the cluster cores (400,000 query segments), full time span, d in {1, 5}. One
step = the query set searched at every d with every index (spatiotemporal, temporal, spatial): the
whole search path (query preparation, schedule, grouping, pair kernel count pass, scan, row
placement / write pass) per search, inputs resident in HBM. Other workloads: --workload
random-walk-1m | dense | tiny | merger-like-2m.

Prints ONE JSON line (rank 0). With --impl reference the CPU oracle is timed instead on the host
cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "seg-pair tests/s & query segs/s, plain vs batched/served; p50/p99 latency"
EXACT_FLOPS = 41     # FP64 flops per exact test of the definition (window, positions, a, b, c, decision)
INTERVAL_FLOPS = 10  # FP64 flops per hit for the roots (sqrt, 2 div, clamps; sqrt and div as 1 each)
# Per-unit counts of the pair kernel from ncu captures of the same kernel sources (hash
# `sources`; a profile of other sources is not used): per exact FP64 test, the FP64-pipe thread
# instructions (sm__thread_inst_executed_pipe_fp64_pred_on.sum / exact tests) at the capture's
# hits per exact test (`hit_ratio`); per candidate test, the warp instructions issued
# (smsp__inst_executed.sum / tests); per exact test, DRAM bytes (dram__bytes_read.sum +
# dram__bytes_write.sum; the gathered FP64 records and the kept hits). The merger-like workload at
# a tenth of the particles (merger-like-2m) stands in for the full one, whose launches are too
# large to capture: the per-unit counts are those of the same kernel at the same hit ratio.
_MERGER_PROFILE = {"fp64_inst_per_exact": 33.84, "warp_inst_per_test": 0.4961,
                   "dram_bytes_per_exact": 62.02, "hit_ratio": 0.8697,
                   "capture": "profiles/k_pair_merger-like-2m_count-pass.md",
                   "sources": "2cf662d8c6ac49b1"}
# the Random-walk 1M workload (filter-bound: the issue slots bind); its DRAM bytes are mostly the
# records the sweep streams, scaled here by the exact tests of the same workload
_RW1M_PROFILE = {"fp64_inst_per_exact": 8.80, "warp_inst_per_test": 0.5090,
                 "dram_bytes_per_exact": 438.6, "hit_ratio": 0.348,
                 "capture": "profiles/k_pair_random-walk-1m_count-pass.md",
                 "sources": "2cf662d8c6ac49b1"}
PAIR_PROFILE = {"merger-like-20m": _MERGER_PROFILE, "merger-like-2m": _MERGER_PROFILE,
                "random-walk-1m": _RW1M_PROFILE}
PAIR_SOURCES = ("ts_search.cuh", "ts_internal.cuh", "ts_device.cuh")


def pair_source_hash(csrc=None):
    """Hash of the pair kernel's sources: its headers and its section of ts_search.cu (from the
    pair kernel banner to the placement kernel)."""
    csrc = csrc or os.path.join(ROOT, "paper_1410_2698_gb300", "csrc")
    h = hashlib.sha256()
    for f in PAIR_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "ts_search.cu"), "rb") as fh:
        text = fh.read()
    a = text.index(b"\n// pair kernel\n")
    b = text.index(b"\n// Rows of the hits the count pass kept", a)
    h.update(text[a:b])
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="merger-like")
    ap.add_argument("--indexes", default="spatiotemporal,temporal,spatial")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="records per work tile (0 = default)")
    ap.add_argument("--pair-blocks", type=int, default=0, help="pair kernel blocks (0 = all)")
    ap.add_argument("--t-bins", type=int, default=0,
                    help="temporal bins of the temporal and spatiotemporal indexes when not "
                         "autotuned (0 = the index's default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="default index parameters, tiles and pair grid instead of the "
                         "autotuner's (which times the batched form before the timed region)")
    ap.add_argument("--tune-sample", type=float, default=0.0,
                    help="fraction of the query trajectories the autotuner times (0 = all, or "
                         "a tenth on workloads of more than 5M database segments)")
    ap.add_argument("--serial-plans", action="store_true",
                    help="one batch plan at a time (automatic when the plans would not fit)")
    ap.add_argument("--served-index", default="spatiotemporal")
    ap.add_argument("--served-requests", type=int, default=200)
    ap.add_argument("--served-max-traj", type=int, default=0,
                    help="largest request, in query trajectories (0 = 5,000 on the merger-like "
                         "database, 500 otherwise)")
    ap.add_argument("--served-inflight", type=int, default=2,
                    help="batches of the served loop on the device at once")
    ap.add_argument("--served-rho", default="0.5,0.9,1.5",
                    help="Poisson arrival rates as multiples of the plain request rate")
    ap.add_argument("--served-only", action="store_true",
                    help="only the served form (its own JSON line) on the workload's database")
    ap.add_argument("--study", action="store_true",
                    help="only the index-parameter study (response vs m, v, g and d) as one JSON "
                         "line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_workload(name, rank):
    from paper_1410_2698_gb300 import workloads
    if name == "random-walk-1m":
        w = workloads.random_walk_1m()
        if rank:
            # each rank searches its own query batch (weak scaling): other query trajectories
            qrng = np.random.Generator(np.random.PCG64(workloads.SEED_BASE + 1 + 1000 + rank))
            q_traj = np.sort(qrng.choice(2500, size=25, replace=False))
            w.queries = workloads._query_from_traj(w.db, 400, q_traj)
        return w
    if name == "tiny":
        return workloads.tiny()
    if name == "dense":
        return workloads.dense()
    if name == "merger-like":
        # each rank searches its own draw of core query trajectories (weak scaling)
        return workloads.merger_like(query_seed_offset=rank)
    if name == "merger-like-2m":  # a tenth of the particles (profiling size)
        return workloads.merger_like(n_per_cluster=5000, n_query_traj=200)
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def device_info(dev):
    """SM count and maximum SM clock of the device (the derived issue peak's unit counts)."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    mhz = measured_peaks().get("sm_max_mhz")
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", f"--id={dev.index or 0}",
                                  "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=10).stdout
            mhz = float(out.split()[0])
        except (OSError, ValueError, IndexError, subprocess.SubprocessError):
            mhz = None
    return {"sms": int(props.multi_processor_count), "sm_max_mhz": mhz, "name": props.name}


def roofline(tot, pair_ms, peaks, workload, dev_info):
    """Roofline of the pair kernel (its count and write passes, timed by the CUDA events its plans
    record around them inside the timed step). The kernel's work runs on two pipes: the FP64 pipe
    (the exact tests; the FP32 filters decide every other candidate) and the issue slots of the SM
    sub-partitions (the FP32 filters' sweep). For each, achieved = the instructions the kernel
    issued for this step's work (per-unit counts from the ncu capture of the same sources, times
    this step's exact tests or candidate tests) / the kernel's time; peak = the FP64 pipe's
    measured instruction rate (the DFMA loop of ts_measure_alu_peaks: TFLOP/s / 2) or the issue
    rate derived from the unit counts (SMs x 4 sub-partitions x 1 warp instruction per clock x the
    maximum SM clock). The bound is the pipe with the larger fraction. Beside it: the algorithmic
    FP64 flops of the definition (41 per exact test, 10 per hit) against the measured DFMA peak,
    and HBM bytes from the capture."""
    t_s = pair_ms / 1e3
    prof = PAIR_PROFILE.get(workload)
    cur = pair_source_hash()
    valid = prof is not None and prof["sources"] == cur
    fp64_inst_peak = peaks["fp64_tflops"] * 1e12 / 2.0
    mhz = dev_info.get("sm_max_mhz") or 0.0
    issue_peak = dev_info["sms"] * 4 * mhz * 1e6
    alg = (tot["n_exact"] * EXACT_FLOPS + tot["n_hits"] * INTERVAL_FLOPS)
    out = {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
           "traffic": None, "kernel": "k_pair (count + write passes)",
           "pair_ms_per_step": pair_ms,
           "work_per_step": {"candidate_tests": tot["n_tests"], "exact_tests": tot["n_exact"],
                             "hits": tot["n_hits"]},
           "algorithmic_fp64": {
               "achieved_tflops": alg / t_s / 1e12 if t_s > 0 else None,
               "peak_tflops": peaks["fp64_tflops"],
               "frac": alg / t_s / 1e12 / peaks["fp64_tflops"] if t_s > 0 else None,
               "note": "41 FP64 flops per exact test and 10 per hit (sqrt and division one "
                       "flop each) against the measured DFMA peak (an FMA two flops)"},
           "profile": prof["capture"] if valid else None,
           "profile_sources": cur}
    if not valid or t_s <= 0 or not mhz:
        out["note"] = ("no ncu capture of the current pair-kernel sources for this workload: "
                       "the pipe fractions are not computed")
        return out
    fp64 = prof["fp64_inst_per_exact"] * tot["n_exact"] / t_s
    issue = prof["warp_inst_per_test"] * tot["n_tests"] / t_s
    pipes = {
        "fp64": {"achieved": fp64 / 1e9, "peak": fp64_inst_peak / 1e9,
                 "frac": fp64 / fp64_inst_peak, "unit": "G FP64 thread-inst/s",
                 "peak_source": "measured: DFMA loop over every SM (ts_measure_alu_peaks), "
                                "TFLOP/s / 2"},
        "issue": {"achieved": issue / 1e9, "peak": issue_peak / 1e9,
                  "frac": issue / issue_peak, "unit": "G warp-inst/s",
                  "peak_source": f"derived: {dev_info['sms']} SMs x 4 sub-partitions x 1 warp "
                                 f"instruction per clock x {mhz:g} MHz"}}
    name = max(pipes, key=lambda k: pipes[k]["frac"])
    top = pipes[name]
    out.update({"achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
                "frac": top["frac"], "pipe": name, "peak_source": top["peak_source"],
                "pipes": pipes,
                "hit_ratio": tot["n_hits"] / max(tot["n_exact"], 1),
                "profile_hit_ratio": prof.get("hit_ratio")})
    if prof.get("dram_bytes_per_exact") is not None:
        launches = max(tot.get("launches", 1), 1)
        out["traffic"] = prof["dram_bytes_per_exact"] * tot["n_exact"] / launches
        out["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum per count-pass "
                               "launch (the write passes sweep no tile when every hit was kept), "
                               "scaled from the capture by this step's exact tests")
        out["algorithmic_bytes"] = {
            "per_exact_test": 64 + 80, "per_hit": 32 + 24,
            "note": "the entry's and the query's FP64 records per exact test (gathered, mostly "
                    "from L2) and a kept hit plus its row per hit; records read by the FP32 "
                    "sweep (32 B, shared by up to 32 queries) not counted"}
    return out


def _timed(args, stream, flush, step, steps=None):
    """Time `steps` calls of step() with CUDA events on the bench stream; the L2 is flushed (a
    256 MB write, finished before the step starts) before every step, outside the events. A step
    that runs on other streams synchronises with the host before it returns, so the events
    bracket all of its work."""
    import torch
    ms = []
    for _ in range(args.steps if steps is None else steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        stream.synchronize()
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def _max_over_ranks(x, world, dev):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1410_2698_gb300 import api
    from paper_1410_2698_gb300.workloads import Segments

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # the bench's own launches (plain searches, L2 flush, step events) go to one side stream;
    # every batch plan runs on a stream of its own
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    w = load_workload(args.workload, rank)
    kinds = [k for k in args.indexes.split(",") if k]
    tuned = {}
    tune_note = None
    if args.autotune:
        # the autotuner times the batched form on this workload's requests (outside the timed
        # region) and caches its choice per workload and GPU; on a large database it times a
        # sample of the query trajectories (the choice is per database and index)
        from paper_1410_2698_gb300 import autotune
        frac = args.tune_sample or (0.1 if w.db.n > 5_000_000 else 1.0)
        tq = w.queries
        if frac < 1.0:
            n_traj = len(w.query_traj_ids)
            per = w.queries.n // n_traj
            keep = max(1, int(round(frac * n_traj)))
            tq = w.queries.take(np.arange(keep * per))
            tune_note = f"timed on {keep} of {n_traj} query trajectories"
        treqs = [(tq, d, w.t_start, w.t_end) for d in w.distances]
        reps = 10 if frac >= 1.0 else 3
        for k in kinds:
            tuned[k] = autotune.tune(w.db, treqs, k, repeats=reps)
    def index_params(k):
        if k in tuned:
            return tuned[k]["index"]
        return {"t_bins": args.t_bins} if args.t_bins and k in ("temporal",
                                                                  "spatiotemporal") else {}

    indexes = {k: api.ts_build_index(w.db, kind=k, **index_params(k)) for k in kinds}
    qdev = {f: torch.from_numpy(getattr(w.queries, f)).to(dev) for f in Segments.FIELDS}
    torch.cuda.synchronize()
    peaks = api.ts_measure_alu_peaks()  # roofline denominators, measured before the timed region
    dinfo = device_info(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    stream = torch.cuda.current_stream()

    # plain form: one ts_search per (index, d)
    def plain_step(collect=None):
        for k in kinds:
            for d in w.distances:
                r = api.ts_search(indexes[k], qdev, d, w.t_start, w.t_end)
                if collect is not None:
                    collect.append((k, d, r.stats))
                r.free()

    warm = []
    for _ in range(max(args.warmup, 0)):
        plain_step(warm)
    rows_per_batch = {k: sum(st["n_hits"] for kk, _, st in warm if kk == k) // max(args.warmup, 1)
                      for k in kinds}
    # a batch's tiles are its requests' tiles (one request per d)
    tiles_per_batch = {k: sum(st["n_tiles"] for kk, _, st in warm if kk == k) //
                       max(args.warmup, 1) for k in kinds}
    # batched form: one reusable plan per index, replayed as a CUDA graph; the distances are the
    # requests of one batch
    reqs = [(qdev, d, w.t_start, w.t_end) for d in w.distances]
    preq = api.prepare_requests(reqs)  # marshalled once for every run of the plans
    # a plan holds its rows (24 B) and the count pass's kept hits (32 B) for max_rows rows
    plan_bytes = sum(56 * max(1 << 20, 2 * rows_per_batch[k]) for k in kinds)
    serial = args.serial_plans or plan_bytes > 60e9

    # grid plans hold one unit per z-run of a query's cells: their count from the schedule
    units = {}
    for k in kinds:
        if k == "spatial":
            units[k] = sum(int(api.ts_schedule(indexes[k], w.queries, d, w.t_start,
                                               w.t_end)[1].sum()) for d in w.distances)
            units[k] += units[k] // 10 + 1024
        else:
            units[k] = 0  # one unit per query (the plan's default)

    def make_plan(k, own_stream, pair_blocks=None):
        rows = (rows_per_batch[k] + rows_per_batch[k] // 20 + (1 << 20)) if serial else \
            max(1 << 20, 2 * rows_per_batch[k])
        if pair_blocks is None:  # an explicit --pair-blocks overrides the tuned grid
            pair_blocks = args.pair_blocks or (tuned[k]["pair_blocks"] if k in tuned else 0)
        return api.BatchPlan(indexes[k], max_requests=len(reqs),
                             max_queries=w.queries.n * len(reqs), max_rows=rows, use_graph=True,
                             stream=0 if own_stream else None,
                             tile_records=tuned[k]["tile_records"] if k in tuned else args.tile,
                             pair_blocks=pair_blocks, max_units=units[k],
                             max_tiles=tiles_per_batch[k] + tiles_per_batch[k] // 10 + 65536)

    batch_stats = []
    alone = []
    plans = {}
    step_pair_blocks = None
    order = list(kinds)  # the order the plans of a step are launched in
    if not serial and args.autotune:
        # the plans of a step overlap on their own streams: the pair grid they share and the
        # order they are launched in are tuned on the overlapped step itself, outside the timed
        # region
        from paper_1410_2698_gb300 import autotune
        step_pair_blocks, order = autotune.tune_overlapped(
            lambda pb: {k: make_plan(k, True, pb) for k in kinds}, kinds, preq,
            tune_grid=not args.pair_blocks)
    if not serial:
        plans = {k: make_plan(k, True, step_pair_blocks) for k in kinds}

        def batched_step(collect=None):
            for k in order:
                plans[k].run(preq, stream=0)  # each plan on its own stream: the plans overlap
            for k in order:
                st = plans[k].wait()
                if st["overflow"]:
                    raise RuntimeError(f"batch plan overflow for {k}")
                if collect is not None:
                    collect.append((k, st))

        for _ in range(max(args.warmup, 0)):
            batched_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = api.ts_kernel_launches()
    per = []
    plain_ms = _timed(args, stream, flush, lambda: plain_step(per))
    l1 = api.ts_kernel_launches()
    if not serial:
        batch_ms = _timed(args, stream, flush, lambda: batched_step(batch_stats))
        l2 = api.ts_kernel_launches()

        # the pair kernel timed alone: the same plans, one at a time on the bench stream (in
        # the overlapped step the events of one plan also see the other plans' kernels)
        def alone_step():
            for k in kinds:
                plans[k].run(preq)
                alone.append((k, plans[k].wait()))

        alone_ms = _timed(args, stream, flush, alone_step, steps=min(args.steps, 20))
    else:
        # one plan at a time (setup outside the timed region): a step's time is the sum of the
        # indexes' step times
        batch_ms = [0.0] * args.steps
        launched = 0
        for k in kinds:
            plan = make_plan(k, False)

            def one(plan=plan, k=k):
                plan.run(preq)
                st = plan.wait()
                if st["overflow"]:
                    raise RuntimeError(f"batch plan overflow for {k}")
                batch_stats.append((k, st))

            for _ in range(max(args.warmup, 0)):
                plan.run(preq)
                plan.wait()
            n0 = len(batch_stats)
            a = api.ts_kernel_launches()
            for i, v in enumerate(_timed(args, stream, flush, one)):
                batch_ms[i] += v
            launched += api.ts_kernel_launches() - a
            alone.extend(batch_stats[n0:])
            plan.free()
        l2 = l1 + launched
        alone_ms = batch_ms
    torch.cuda.synchronize()
    clk = clocks.stop()
    plain_total = _max_over_ranks(float(sum(plain_ms)), world, dev)
    batch_total = _max_over_ranks(float(sum(batch_ms)), world, dev)

    tot = {k: 0 for k in ("n_tests", "n_exact", "n_hits", "n_qsegs")}
    pair_ms = 0.0
    breakdown = {}
    for k, d, st in per:
        for key in tot:
            tot[key] += st[key]
        pair_ms += st["ms_count_pass"] + st["ms_write_pass"]
        b = breakdown.setdefault(f"{k}@d={d:g}", {"tests": 0, "hits": 0, "pair_ms": 0.0,
                                                  "exact": 0, "subbin_queries": 0, "chunks": 0,
                                                  "dense_chunks": 0, "sparse_visits": 0,
                                                  "stage2": 0})
        b["chunks"] += st["n_chunks"]
        b["dense_chunks"] += st["n_dense"]
        b["sparse_visits"] += st["n_sparse"]
        b["stage2"] += st["n_stage2"]
        b["tests"] += st["n_tests"]
        b["hits"] += st["n_hits"]
        b["exact"] += st["n_exact"]
        b["subbin_queries"] += st["n_subbin"]
        b["pair_ms"] += st["ms_count_pass"] + st["ms_write_pass"]
    for b in breakdown.values():
        for key in ("tests", "hits", "exact", "subbin_queries", "chunks", "dense_chunks",
                    "sparse_visits", "stage2"):
            b[key] //= max(args.steps, 1)
        b["pair_ms"] /= max(args.steps, 1)
    btot = {"n_qsegs": 0, "n_tests": 0, "n_hits": 0, "n_exact": 0}
    for _, st in batch_stats:
        for key in btot:
            btot[key] += st["stats"][key]
    assert btot["n_hits"] == tot["n_hits"], "batched and plain forms disagree"
    atot = {"n_qsegs": 0, "n_tests": 0, "n_hits": 0, "n_exact": 0}
    apair_ms = 0.0
    per_index = {}
    for k, st in alone:
        for key in atot:
            atot[key] += st["stats"][key]
        ms = st["stats"]["ms_count_pass"] + st["stats"]["ms_write_pass"]
        apair_ms += ms
        e = per_index.setdefault(k, {"pair_ms": 0.0, "tests": 0, "tiles": 0, "groups": 0})
        e["pair_ms"] += ms
        e["tests"] += st["stats"]["n_tests"]
        e["tiles"] += st["stats"]["n_tiles"]
        e["groups"] += st["stats"]["n_groups"]
    n_alone = max(len(alone_ms), 1)
    for e in per_index.values():
        for key in e:
            e[key] = e[key] / n_alone
    # roofline of the dominant kernel: the batched pair kernel (count + write passes), timed by
    # the CUDA events each plan records around its passes on its stream. With the plans run one
    # at a time these are the timed headline step's own events; with overlapped plans (where a
    # plan's events also span the other plans' kernels) a loop of the same plans one at a time.
    step_tot = {k: v / n_alone for k, v in atot.items()}  # per step
    step_tot["launches"] = len(kinds)  # count passes (one per plan)
    roof = roofline(step_tot, apair_ms / n_alone, peaks, w.name, dinfo)
    if serial:
        roof["timed_form"] = ("batched, the timed headline step itself (plans one at a time; "
                              "CUDA events of each plan around its pair-kernel passes)")
    else:
        roof["timed_form"] = "batched, one plan at a time (a loop of the headline step's plans)"
    roof["pair_kernel_share"] = apair_ms / sum(alone_ms) if alone_ms else None
    roof["per_index"] = per_index
    # whole-job aggregates (every rank processes the same amount of work)
    value = btot["n_qsegs"] * world / (batch_total / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "query segs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: " + STAND_IN.get(w.name.split("-")[0], "seeded trajectories"),
        "config": {"workload": f"{w.name}: {w.db.n} db segments, {w.queries.n} query segments, "
                               f"d in {list(w.distances)}, indexes {kinds}",
                   "form": "batched: per index one reusable plan replayed as a CUDA graph, the "
                           "distances are the requests of one batch",
                   "l2": "flushed (256 MB write) before every timed step",
                   "tile_records": {k: (tuned[k]["tile_records"] if k in tuned else
                                        (args.tile or 256)) for k in kinds},
                   "pair_blocks": {k: (step_pair_blocks if step_pair_blocks is not None else
                                       (args.pair_blocks or (tuned[k]["pair_blocks"]
                                                             if k in tuned else 0)))
                                   or "all resident" for k in kinds},
                   "gpu": f"{dinfo['name']}, {dinfo['sms']} SMs"},
        "tests_per_s": btot["n_tests"] * world / (batch_total / 1e3),
        # every clipped query segment against every database segment, per second (what an
        # all-pairs search would have to evaluate; a label, not a count of work done)
        "brute_equivalent_pairs_per_s": btot["n_qsegs"] * w.db.n * world / (batch_total / 1e3),
        "hits_per_step": btot["n_hits"] // max(args.steps, 1),
        "gpu_launches": int(l2 - l1),
        "clocks": clk,
        "roofline": roof,
        "plain": {"value": tot["n_qsegs"] * world / (plain_total / 1e3), "unit": "query segs/s",
                  "ms_per_step": plain_total / args.steps,
                  "tests_per_s": tot["n_tests"] * world / (plain_total / 1e3),
                  "gpu_launches": int(l1 - l0),
                  "pair_kernel_share": pair_ms / plain_total if plain_total else None,
                  "form": "one ts_search per index and d"},
        "breakdown": breakdown,
    }
    line["config"]["plans"] = "one at a time" if serial else "resident together, overlapped"
    if not serial:
        line["config"]["launch_order"] = order
    line["config"]["index_params"] = {k: _index_params(indexes[k]) for k in kinds}
    if tuned:
        line["config"]["autotuned"] = {k: {"index": v["index"], "tile_records": v["tile_records"],
                                           "pair_blocks": v["pair_blocks"]}
                                       for k, v in tuned.items()}
        if tune_note:
            line["config"]["autotune_sample"] = tune_note
    if not args.no_e2e:
        most = max(rows_per_batch.values()) if rows_per_batch else 0
        if serial:
            # the end-to-end step holds the plans together when the device has room for them at
            # their exact row counts, runs them one after another on one stream and copies the
            # rows of one plan to the host while the next ones compute; else one plan at a time
            e2e_plans = {}
            try:
                for k in kinds:
                    e2e_plans[k] = make_plan(k, True)
            except api.TsError:
                for pl in e2e_plans.values():
                    pl.free()
                e2e_plans = None
            if e2e_plans:
                line["e2e"] = run_e2e(args, api, w, e2e_plans, order, max_rows=most,
                                      sequential=True)
                line["e2e"]["plans"] = ("resident together, run one after another on one stream "
                                        "(each plan's rows copied while the next plans run)")
                for pl in e2e_plans.values():
                    pl.free()
            else:
                line["e2e"] = run_e2e(args, api, w, None, kinds, make_plan, most)
                line["e2e"]["plans"] = "one at a time"
        else:
            line["e2e"] = run_e2e(args, api, w, plans, order, max_rows=most)
    if not args.no_served and rank == 0:
        sk = args.served_index
        sidx = indexes[sk] if sk in indexes else api.ts_build_index(w.db, kind=sk)
        # the served stream's requests run at the tuned tile size of the served index
        line["served"] = run_served(args, api, w, sidx,
                                    tile=tuned[sk]["tile_records"] if sk in tuned else 0)
    if world > 1:
        dist.barrier()
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w)
    for pl in plans.values():
        pl.free()
    for idx in indexes.values():
        idx.free()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


STAND_IN = {
    "merger": "two Plummer-sphere clusters on ballistic-plus-jitter paths (stand-in for the "
              "paper's Merger N-body data)",
    "random": "seeded random walks (stand-in for the paper's Random-1M)",
    "dense": "seeded random walks in a box with reflecting walls (stand-in for the paper's "
             "Random-dense)",
    "tiny": "seeded random walks (parity case)",
}


def _index_params(index):
    info = index.info()
    kind = {0: "brute", 1: "spatial", 2: "temporal", 3: "spatiotemporal"}[int(info["kind"])]
    if kind == "temporal":
        return {"t_bins": int(info["t_bins"])}
    if kind == "spatiotemporal":
        return {"t_bins": int(info["t_bins"]), "sub_bins": [int(v) for v in info["sub_bins"]]}
    if kind == "spatial":
        return {"grid_cells": int(info["grid_cells"])}
    return {}


E2E_CHUNK_ROWS = 1 << 27  # rows per read of the end-to-end step (3 GB of pinned host memory)


def _pinned_rows(n):
    """Pinned host buffers for n result rows (numpy views of page-locked torch tensors)."""
    import torch
    mk = lambda dt: torch.empty(max(n, 1), dtype=dt, pin_memory=True)  # noqa: E731
    t = {"q_idx": mk(torch.int32), "e_idx": mk(torch.int32), "t_in": mk(torch.float64),
         "t_out": mk(torch.float64)}
    views = {k: v.numpy().view(np.uint32) if k in ("q_idx", "e_idx") else v.numpy()
             for k, v in t.items()}
    return views, t


def run_e2e(args, api, w, plans, kinds, make_plan=None, max_rows=0, sequential=False):
    """The batched step through the C ABI with HOST buffers: the query columns live in pinned
    host memory (the plans read them from there) and every result row is read back into pinned
    host memory inside the timed region (wall clock, the stream synchronised on both sides), in
    chunks of at most E2E_CHUNK_ROWS rows through one pinned buffer (the host memory it holds stays
    bounded whatever the step's rows, also with one process per GPU). With make_plan (plans that
    do not fit together) each index's plan is created, timed over the steps and released in
    turn. With `sequential`, resident plans run one after another on one stream (large plans: the
    first one's rows are ready a third of the way into the step and each plan's rows are read
    while the next ones compute); else each on its own stream, overlapped, as in the timed
    step."""
    import torch
    from paper_1410_2698_gb300.workloads import Segments
    qhost = {f: torch.from_numpy(np.ascontiguousarray(getattr(w.queries, f))).pin_memory()
             for f in Segments.FIELDS}
    reqs = api.prepare_requests([(qhost, d, w.t_start, w.t_end) for d in w.distances])
    rows_out, keep = _pinned_rows(min(max_rows, E2E_CHUNK_ROWS))

    def read_rows(plan, total):
        """Every row of the plan's last run, chunk by chunk; returns the bytes read."""
        n = 0
        for first in range(0, total, E2E_CHUNK_ROWS):
            n += plan.copy_rows(first, min(E2E_CHUNK_ROWS, total - first), rows_out)
        return n
    if make_plan is not None:
        total_ms, copy_ms, h2d, d2h, qsegs = 0.0, 0.0, 0, 0, 0
        copies = []
        steps = max(1, min(args.steps, 5))
        for k in kinds:
            plan = make_plan(k, False)
            plan.run(reqs)
            plan.wait()  # warm-up
            for _ in range(steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                plan.run(reqs)
                st = plan.wait()
                t1 = time.perf_counter()
                d2h += read_rows(plan, st["rows"])  # every request's rows
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                total_ms += (t2 - t0) * 1e3
                copy_ms += (t2 - t1) * 1e3
                copies.append(round((t2 - t1) * 1e3, 1))
                qsegs += st["stats"]["n_qsegs"]
                h2d += 8 * 8 * w.queries.n * reqs.n
            plan.free()
        return {"value": qsegs / (total_ms / 1e3), "unit": "query segs/s",
                "h2d_bytes_per_step": h2d // steps, "d2h_bytes_per_step": d2h // steps,
                "steps": steps, "host_buffers": "pinned",
                "rows_copy_ms_per_step": copy_ms / steps,
                "rows_copy_gbs": d2h / (copy_ms / 1e3) / 1e9 if copy_ms else None,
                "rows_copy_ms": copies}
    ms = []
    h2d = d2h = qsegs = 0
    copy_ms = 0.0
    # a step is seconds long on the largest workloads: at most 5 timed steps after one warm-up
    steps = args.steps if w.db.n <= 5_000_000 else max(1, min(args.steps, 5))
    seq = torch.cuda.Stream() if sequential else None
    for s in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d_s = d2h_s = q_s = 0
        for k in kinds:
            # (stream 0: each plan on its own stream)
            plans[k].run(reqs, stream=seq.cuda_stream if seq is not None else 0)
        for k in kinds:
            st = plans[k].wait()  # this plan's run only
            q_s += st["stats"]["n_qsegs"]
            c0 = time.perf_counter()
            d2h_s += read_rows(plans[k], st["rows"])  # every request's rows
            if s > 0:
                copy_ms += (time.perf_counter() - c0) * 1e3
            h2d_s += 8 * 8 * w.queries.n * reqs.n
        torch.cuda.synchronize()
        if s > 0:  # the first pass is warm-up
            ms.append((time.perf_counter() - t0) * 1e3)
            h2d, d2h, qsegs = h2d_s, d2h_s, q_s
    t = sum(ms) / 1e3
    return {"value": qsegs * len(ms) / t, "unit": "query segs/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "host_buffers": "pinned", "steps": len(ms),
            "rows_copy_ms_per_step": copy_ms / max(len(ms), 1)}


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def served_max_traj(args, w):
    return args.served_max_traj or (5000 if w.name.startswith("merger") else 500)


def run_served(args, api, w, index, tile=0):
    """The served form on the resident database: a stream of requests (each a set of query
    trajectory runs with its own interval and d, query arrays on the host) through the request
    loop, against one plain ts_search per request. Passes over the same requests: plain (one
    after another, each synchronous), served at saturation (all submitted at once) and served
    with Poisson arrivals at rho x the plain request rate for every rho of --served-rho.
    Latency = completion - arrival (the server's clock); every result is released after its
    count is read."""
    import threading
    from paper_1410_2698_gb300 import workloads
    max_traj = served_max_traj(args, w)
    stream = workloads.served_stream(w, n_requests=args.served_requests, rate_per_s=1.0,
                                     max_traj=max_traj)
    qsegs = sum(r.queries.n for r in stream)
    max_q = max(r.queries.n for r in stream)
    # plain: one synchronous search per request (after two warm-up searches)
    for r in stream[:2]:
        api.ts_search(index, r.queries, r.d, r.t_start, r.t_end).free()
    lat_plain, rows_plain, max_rows = [], 0, 0
    t0 = time.perf_counter()
    for r in stream:
        a = time.perf_counter()
        res = api.ts_search(index, r.queries, r.d, r.t_start, r.t_end)
        rows_plain += res.count
        max_rows = max(max_rows, res.count)
        res.free()
        lat_plain.append((time.perf_counter() - a) * 1e3)
    plain_s = time.perf_counter() - t0
    mu_plain = len(stream) / plain_s

    def plain_arrivals(arrivals):
        """One plain search per request in arrival order on one worker (a FIFO server of plain
        launches): latency = completion - arrival, queueing included."""
        import queue
        qu = queue.Queue()
        lat = [0.0] * len(stream)
        start = time.perf_counter()

        def worker():
            while True:
                item = qu.get()
                if item is None:
                    return
                i, t_arr = item
                r = stream[i]
                api.ts_search(index, r.queries, r.d, r.t_start, r.t_end).free()
                lat[i] = (time.perf_counter() - t_arr) * 1e3

        th = threading.Thread(target=worker)
        th.start()
        for i in range(len(stream)):
            dt = start + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            qu.put((i, start + arrivals[i]))
        qu.put(None)
        th.join()
        return time.perf_counter() - start, lat
    srv = api.Server(index, max_batch_requests=64, max_batch_queries=max(1 << 20, 2 * max_q),
                     max_batch_rows=max(1 << 25, 2 * max_rows),
                     max_inflight=args.served_inflight, use_graph=True, linger_us=200,
                     tile_records=tile)
    rhos = [float(x) for x in str(args.served_rho).split(",") if x]
    try:
        def serve(arrivals):
            tickets = [None] * len(stream)
            start = time.perf_counter()

            def submitter():
                for i, r in enumerate(stream):
                    if arrivals is not None:
                        dt = start + arrivals[i] - time.perf_counter()
                        if dt > 0:
                            time.sleep(dt)
                    tickets[i] = srv.submit(r.queries, r.d, r.t_start, r.t_end)

            th = threading.Thread(target=submitter)
            th.start()
            lat, rows, sizes = [], 0, []
            for i in range(len(stream)):
                while tickets[i] is None:
                    time.sleep(1e-5)
                res, tm = srv.wait(tickets[i], timeout_ms=600000)
                rows += res.count
                res.free()
                lat.append((tm["done_us"] - tm["submit_us"]) / 1e3)
                sizes.append(tm["batch_requests"])
            th.join()
            return time.perf_counter() - start, lat, rows, sizes

        serve(None)  # warm-up: plans captured as graphs
        sat_s, lat_sat, rows_sat, sizes_sat = serve(None)
        poisson = []
        for rho in rhos:
            lam = rho * mu_plain
            arrivals = [r.arrival_s / lam for r in stream]  # the stream's gaps are at rate 1
            poi_s, lat_poi, rows_poi, sizes_poi = serve(arrivals)
            if rows_poi != rows_plain:
                raise RuntimeError("served and plain forms disagree on the result count")
            pl_s, lat_pl = plain_arrivals(arrivals)
            poisson.append({"rho": rho, "arrival_rate_req_s": lam,
                            "qsegs_per_s": qsegs / poi_s, "p50_ms": _pct(lat_poi, 50),
                            "p99_ms": _pct(lat_poi, 99),
                            "mean_batch_requests": float(np.mean(sizes_poi)),
                            "plain": {"qsegs_per_s": qsegs / pl_s, "p50_ms": _pct(lat_pl, 50),
                                      "p99_ms": _pct(lat_pl, 99),
                                      "form": "the same arrivals, one plain search per request "
                                              "in arrival order (queueing included)"}})
    finally:
        srv.close()
    if rows_plain != rows_sat:
        raise RuntimeError("served and plain forms disagree on the result count")
    return {
        "index": index_kind_name(index), "max_inflight": args.served_inflight,
        "requests": len(stream), "query_segs": qsegs, "rows": rows_plain,
        "workload": f"{len(stream)} requests on the resident {w.name} database: 1-{max_traj} "
                    f"query trajectory runs (log-uniform) of 10-200 segments, interval = the "
                    f"runs' span, d log-uniform in [0.5, 10]; query arrays on the host",
        "max_request_rows": max_rows,
        "plain": {"qsegs_per_s": qsegs / plain_s, "req_per_s": mu_plain,
                  "p50_ms": _pct(lat_plain, 50), "p99_ms": _pct(lat_plain, 99),
                  "form": "one synchronous ts_search per request"},
        "saturated": {"qsegs_per_s": qsegs / sat_s, "req_per_s": len(stream) / sat_s,
                      "p50_ms": _pct(lat_sat, 50), "p99_ms": _pct(lat_sat, 99),
                      "mean_batch_requests": float(np.mean(sizes_sat)),
                      "form": "every request submitted at once"},
        "poisson": poisson,
    }


def index_kind_name(index):
    return {0: "brute", 1: "spatial", 2: "temporal", 3: "spatiotemporal"}.get(
        int(index.info()["kind"]), "?")


def cpu_model():
    """The host CPU's model name (lscpu; /proc/cpuinfo or the platform as fallbacks)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(w, budget_s=8.0):
    """The oracle as it stands, on all host cores (OpenMP), on a bounded sample of the
    workload's query segments at every d; reported in query segs/s."""
    import oracle
    from paper_1410_2698_gb300.workloads import Segments
    threads = os.cpu_count() or 1
    nq = w.queries.n
    take = min(nq, 500)
    spent = 0.0
    qsegs = 0
    tests = 0
    rounds = 0
    while spent < budget_s and take <= nq:
        sub = w.queries.take(np.arange(take))
        t0 = time.perf_counter()
        for d in w.distances:
            _, nt, nqs = oracle.search_count(w.db, sub, w.t_start, w.t_end, d, threads=threads)
            qsegs += nqs
            tests += nt
        spent += time.perf_counter() - t0
        rounds += 1
        if take == nq:
            break
        take = min(nq, take * 2)
    out = {"value": qsegs / spent, "unit": "query segs/s", "cores": threads, "kind": "oracle",
           "cpu": f"{cpu_model()} ({platform.machine()}, {threads} threads)",
           "tests_per_s": tests / spent,
           "sample": f"{rounds} passes over the first up-to-{take} query segments x "
                     f"{len(w.distances)} distances ({spent:.1f} s of CPU time)"}
    # the same oracle on one core, on a smaller sample (the first distance only)
    take1 = min(nq, 200)
    sub = w.queries.take(np.arange(take1))
    spent1 = qsegs1 = tests1 = 0
    while spent1 < budget_s / 4:
        t0 = time.perf_counter()
        _, nt, nqs = oracle.search_count(w.db, sub, w.t_start, w.t_end, w.distances[0], threads=1)
        spent1 += time.perf_counter() - t0
        qsegs1 += nqs
        tests1 += nt
    out["single_thread"] = {"value": qsegs1 / spent1, "unit": "query segs/s", "cores": 1,
                            "tests_per_s": tests1 / spent1,
                            "sample": f"the first {take1} query segments at d = "
                                      f"{w.distances[0]:g} ({spent1:.1f} s)"}
    out["rtree"] = rtree_baseline(w, threads, budget_s=budget_s / 2)
    return out


def rtree_baseline(w, threads, rs=(1, 2, 4), budget_s=4.0):
    """The CPU R-tree (the paper's CPU comparator: r consecutive segments of a trajectory per 4-D
    box, STR-packed, OpenMP queries, the oracle's pair test) on all host cores, for every r, on a
    growing prefix of the query segments at every d until ~budget_s of queries; the build is
    timed separately (not part of the rate, as the GPU index build is not)."""
    import oracle
    res = {"kind": "rtree", "unit": "query segs/s", "cores": threads,
           "cpu": f"{cpu_model()} ({platform.machine()}, {threads} threads)", "by_r": {}}
    best = None
    nq = w.queries.n
    for r in rs:
        t0 = time.perf_counter()
        tree = oracle.RTree(w.db, r)
        build_s = time.perf_counter() - t0
        take, spent, qsegs, tests, passes = min(nq, 500), 0.0, 0, 0, 0
        while spent < budget_s:
            sub = w.queries.take(np.arange(take))
            t0 = time.perf_counter()
            for d in w.distances:
                _, nt, nqs = tree.count(sub, w.t_start, w.t_end, d, threads=threads)
                qsegs += nqs
                tests += nt
            spent += time.perf_counter() - t0
            passes += 1
            take = min(nq, take * 2)
        tree.free()
        v = qsegs / spent
        res["by_r"][str(r)] = {"value": v, "tests_per_s": tests / spent, "build_s": build_s,
                               "sample": f"{passes} passes over query-segment prefixes up to "
                                         f"{sub.n} x {len(w.distances)} distances "
                                         f"({spent:.1f} s)"}
        if best is None or v > best[1]:
            best = (r, v)
    res["value"] = best[1]
    res["best_r"] = best[0]
    return res


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    w = load_workload(args.workload, 0)
    threads = os.cpu_count() or 1
    # a bounded sample: ~1-2 s of the host's cores per step on every workload
    sample = w.queries.take(np.arange(min(w.queries.n, 800 if w.db.n <= 2_000_000 else 400)))
    for _ in range(max(args.warmup, 0)):
        oracle.search_count(w.db, sample.take(np.arange(50)), w.t_start, w.t_end, w.distances[0],
                            threads=threads)
    total = 0.0
    qsegs = 0
    tests = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for d in w.distances:
            _, nt, nq = oracle.search_count(w.db, sample, w.t_start, w.t_end, d, threads=threads)
            qsegs += nq
            tests += nt
        total += time.perf_counter() - t0
    value = qsegs / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "query segs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.db.n} db segments, sample of {sample.n} of "
                                   f"{w.queries.n} query segments, d in {list(w.distances)}"},
            "cpu_baseline": {"value": value, "unit": "query segs/s", "cores": threads,
                             "kind": "oracle", "cpu": f"{cpu_model()} ({platform.machine()})",
                             "sample": f"{sample.n} query segments x {len(w.distances)} d per step"},
            "e2e": {"value": value, "unit": "query segs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "tests_per_s": tests / total}
    print(json.dumps(line), flush=True)


def run_served_only(args):
    """The served form alone on the workload's database: one JSON line (rank 0)."""
    import torch
    from paper_1410_2698_gb300 import api
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    w = load_workload(args.workload, 0)
    idx = api.ts_build_index(w.db, kind=args.served_index)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    served = run_served(args, api, w, idx)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": served["saturated"]["qsegs_per_s"], "unit": "query segs/s",
            "n_gpus": 1, "form": "served (saturated); plain and Poisson beside it",
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.db.n} db segments (resident), "
                                   f"{args.served_index} index; " + served["workload"]},
            "clocks": clk, "served": served}
    print(json.dumps(line), flush=True)
    idx.free()


def run_study(args):
    """The index-parameter study on the workload (plain searches, device-resident queries)."""
    import torch
    from paper_1410_2698_gb300 import api, autotune
    from paper_1410_2698_gb300.workloads import Segments
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    w = load_workload(args.workload, 0)
    dev = torch.device("cuda", local)
    qdev = {f: torch.from_numpy(getattr(w.queries, f)).to(dev) for f in Segments.FIELDS}
    kinds = [k for k in args.indexes.split(",") if k]
    clocks = ClockSampler(local)
    clocks.start()
    rows = autotune.study(w.db, qdev, w.distances, w.t_start, w.t_end, kinds=kinds)
    clk = clocks.stop()
    print(json.dumps({"study": "index granularity", "workload": f"{w.name}: {w.db.n} db segments, "
                      f"{w.queries.n} query segments", "clocks": clk, "records": rows}),
          flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.study:
        run_study(args)
    elif args.served_only:
        run_served_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
