"""Host-side logic that needs no GPU: request marshalling for batch plans, the benchmark's
roofline arithmetic and the gating of its DRAM-traffic figure on the pair kernel's sources."""
import ctypes
import os
import re
import sys

import numpy as np

from paper_1410_2698_gb300 import api, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_prepared_requests_point_at_the_callers_columns():
    w = workloads.tiny()
    q = w.queries
    reqs = [(q, 1.0, 0.0, 70.0), (q, 5.0, 3.0, 60.0, 1000)]
    prep = api.prepare_requests(reqs)
    assert prep.n == 2
    for r, (_, d, ts, te, *mr) in enumerate(reqs):
        s, p = prep.segs[r], prep.qps[r]
        assert s.n == q.n and s.on_host == 1
        # the marshalled columns are the caller's arrays, not copies
        assert ctypes.cast(s.x0, ctypes.c_void_p).value == q.x0.ctypes.data
        assert ctypes.cast(s.t1, ctypes.c_void_p).value == q.t1.ctypes.data
        assert (p.d, p.t_start, p.t_end) == (d, ts, te)
        assert p.max_results == (mr[0] if mr else 0)


def test_roofline_picks_the_busier_pipe_from_the_profile(monkeypatch):
    dev = {"sms": 152, "sm_max_mhz": 2070.0, "name": "GB300"}
    peaks = {"fp32_tflops": 78.5, "fp64_tflops": 1.057}
    fp64_peak = 1.057e12 / 2  # DFMA thread-instructions per second
    issue_peak = 152 * 4 * 2070e6  # warp instructions per second
    # without a capture of the current sources: no pipe fractions, the algorithmic figure only
    monkeypatch.setattr(bench, "PAIR_PROFILE", {})
    r = bench.roofline({"n_tests": 1e9, "n_exact": 1e8, "n_hits": 5e7}, 100.0, peaks, "w", dev)
    assert r["frac"] is None and r["bound"] == "alu"
    alg = (41 * 1e8 + 10 * 5e7) / 0.1 / 1e12
    assert abs(r["algorithmic_fp64"]["achieved_tflops"] - alg) < 1e-12
    assert abs(r["algorithmic_fp64"]["frac"] - alg / 1.057) < 1e-12
    # FP64-dominated: 1e8 exact tests x 60 FP64 instructions in 100 ms
    prof = {"fp64_inst_per_exact": 60.0, "warp_inst_per_test": 0.5, "hit_ratio": 0.5,
            "dram_bytes_per_exact": 100.0, "capture": "profiles/x.md",
            "sources": bench.pair_source_hash()}
    monkeypatch.setattr(bench, "PAIR_PROFILE", {"w": prof})
    tot = {"n_tests": 1e9, "n_exact": 1e8, "n_hits": 5e7, "launches": 2}
    r = bench.roofline(tot, 100.0, peaks, "w", dev)
    assert r["pipe"] == "fp64"
    assert abs(r["frac"] - 60 * 1e8 / 0.1 / fp64_peak) < 1e-12
    assert abs(r["pipes"]["issue"]["frac"] - 0.5 * 1e9 / 0.1 / issue_peak) < 1e-12
    assert abs(r["achieved"] * 1e9 - 60 * 1e8 / 0.1) < 1e-3
    assert r["traffic"] == 100.0 * 1e8 / 2
    # issue-dominated: many candidates, few exact tests
    tot = {"n_tests": 1e11, "n_exact": 1e6, "n_hits": 1e5, "launches": 2}
    r = bench.roofline(tot, 100.0, peaks, "w", dev)
    assert r["pipe"] == "issue"
    assert abs(r["frac"] - 0.5 * 1e11 / 0.1 / issue_peak) < 1e-12
    # a profile of other sources is not used
    monkeypatch.setattr(bench, "PAIR_PROFILE", {"w": dict(prof, sources="0" * 16)})
    assert bench.roofline(tot, 100.0, peaks, "w", dev)["frac"] is None


def test_profile_figures_are_keyed_to_the_pair_kernel_sources(tmp_path):
    csrc = os.path.join(ROOT, "paper_1410_2698_gb300", "csrc")
    h = bench.pair_source_hash()
    assert h == bench.pair_source_hash(csrc) and len(h) == 16
    # a change inside the pair kernel's section changes the hash; one outside it does not
    for f in bench.PAIR_SOURCES + ("ts_search.cu",):
        with open(os.path.join(csrc, f), "rb") as src:
            (tmp_path / f).write_bytes(src.read())
    text = (tmp_path / "ts_search.cu").read_bytes()
    a = text.index(b"\n// pair kernel\n")
    (tmp_path / "ts_search.cu").write_bytes(text[:a] + b"\n// (outside)\n" + text[a:])
    assert bench.pair_source_hash(str(tmp_path)) == h
    b = text.index(b"__global__", a)
    (tmp_path / "ts_search.cu").write_bytes(text[:b] + b"/* inside */ " + text[b:])
    assert bench.pair_source_hash(str(tmp_path)) != h


def test_every_profile_entry_names_its_committed_capture():
    """Each per-unit profile the roofline uses points at a summary under profiles/ that records
    the same pair-kernel sources hash and the same per-unit figures, so the constants and their
    evidence cannot drift apart."""
    for name, prof in bench.PAIR_PROFILE.items():
        path = os.path.join(ROOT, prof["capture"])
        assert os.path.isfile(path), (name, path)
        text = open(path).read()
        assert prof["sources"] in text, (name, prof["sources"])
        bold = [float(x) for x in re.findall(r"\*\*([0-9]+(?:\.[0-9]+)?)", text)]
        for key in ("fp64_inst_per_exact", "warp_inst_per_test", "dram_bytes_per_exact"):
            assert any(abs(x - prof[key]) < 1e-9 for x in bold), (name, key, prof[key], bold)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the CPU oracle on a bounded sample) prints one JSON line with
    the benchmark's keys, its end-to-end entry and the CPU baseline that describes it."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "tiny", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "cpu_baseline"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "workload" in line["config"]


def test_overlapped_step_tuning_picks_the_fastest_grid_then_order():
    from paper_1410_2698_gb300 import autotune

    class FakePlan:
        live = 0

        def __init__(self, pb):
            self.pb = pb
            FakePlan.live += 1

        def free(self):
            FakePlan.live -= 1

    kinds = ["spatiotemporal", "temporal", "spatial"]
    grid_cost = {0: 5.0, 266: 3.0, 228: 2.0, 190: 4.0, 152: 6.0}
    seen = []

    def timer(plans, requests, order):
        pb = next(iter(plans.values())).pb
        seen.append((pb, tuple(order)))
        # the grid is timed in the given order; then the order matters (temporal first best)
        return grid_cost[pb] + (0.0 if order[0] == "temporal" else 1.0) + 0.1 * order.index(
            "spatial")

    # the grids follow the SM count: all resident, then 1.75 / 1.5 / 1.25 / 1 blocks per SM
    assert autotune.step_grids(152) == (0, 266, 228, 190, 152)
    assert autotune.step_grids(148) == (0, 259, 222, 185, 148)
    pb, order = autotune.tune_overlapped(lambda pb: {k: FakePlan(pb) for k in kinds}, kinds,
                                         None, grids=autotune.step_grids(152), timer=timer)
    assert pb == 228
    assert order[0] == "temporal" and order == ["temporal", "spatial", "spatiotemporal"]
    assert FakePlan.live == 0  # every plan made for a trial was freed
    assert len(seen) == 5 + 6
    # with the grid given, only the order is tuned (plans made with pair_blocks None)
    seen.clear()
    pb, order = autotune.tune_overlapped(lambda pb: {k: FakePlan(228 if pb is None else pb)
                                                      for k in kinds}, kinds, None,
                                         tune_grid=False, timer=timer)
    assert pb is None and len(seen) == 6 and order[0] == "temporal"
