"""Multi-rank query sharding on the CPU: two gloo ranks each search their share of the query
trajectories (with the oracle; no GPU) and gather; the merged result must equal the search of the
whole query set. Covers the host-side logic of the multi-GPU path (replicated index, queries
partitioned, no exchange besides the result gather)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    from paper_1410_2698_gb300 import shard, workloads
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    w = workloads.tiny()
    seg_per = w.queries.n // len(w.query_traj_ids)
    traj_first = np.arange(len(w.query_traj_ids)) * seg_per
    mine, off = shard.shard_queries(w.queries, traj_first, rank, world)
    res = oracle.search(w.db, mine, w.t_start, w.t_end, 5.0)
    merged = shard.gather_results({k: res[k] for k in ("q_idx", "e_idx", "t_in", "t_out")}, off)
    if rank == 0:
        full = oracle.search(w.db, w.queries, w.t_start, w.t_end, 5.0)
        ok = all(np.array_equal(merged[k], full[k]) for k in ("q_idx", "e_idx", "t_in", "t_out"))
        with open(os.path.join(out_dir, "ok"), "w") as f:
            f.write("1" if ok and mine.n < w.queries.n else "0")
    dist.destroy_process_group()


def test_two_rank_sharding_matches_single_search(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    assert (tmp_path / "ok").read_text() == "1"


def test_shard_ranges_cover_without_splitting_trajectories():
    from paper_1410_2698_gb300 import shard
    first = np.array([0, 5, 6, 20, 21, 40])
    for world in (1, 2, 3, 4, 7):
        rng = shard.shard_ranges(first, 50, world)
        assert rng[0][0] == 0 and rng[-1][1] == 50
        for (a, b), (c, d) in zip(rng, rng[1:]):
            assert b == c
        for a, b in rng:
            assert a in set(first.tolist()) | {50}


def _timing_rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    # every rank times its own share; the job's time is the slowest rank's
    t = bench._max_over_ranks(10.0 + rank, world, torch.device("cpu"))
    with open(os.path.join(out_dir, f"t{rank}"), "w") as f:
        f.write(repr(t))
    dist.destroy_process_group()


def test_bench_takes_the_slowest_rank_time(tmp_path):
    port = _free_port()
    mp.start_processes(_timing_rank, args=(3, port, str(tmp_path)), nprocs=3, join=True,
                       start_method="spawn")
    for r in range(3):
        assert float((tmp_path / f"t{r}").read_text()) == 12.0
