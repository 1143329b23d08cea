"""Query sharding across GPUs: one process per GPU, the database index replicated on every GPU,
the query trajectories split between ranks, results merged on the host. Query segments are
independent, so the search needs no exchange between ranks; only the (variable-size) results are
gathered.

Host-side logic only (no device work): it is exercised with gloo ranks on the CPU.
"""
from __future__ import annotations

import numpy as np

from .workloads import Segments


def shard_ranges(traj_first: np.ndarray, n_segments: int, world: int):
    """Split trajectories (first segment index of each, ascending) into `world` contiguous ranges
    of roughly equal segment counts. Returns a list of (seg_lo, seg_hi) per rank; trajectories are
    never split."""
    traj_first = np.asarray(traj_first, dtype=np.int64)
    bounds = np.append(traj_first, n_segments)
    out = []
    start_t = 0
    for r in range(world):
        target = (r + 1) * n_segments / world
        end_t = int(np.searchsorted(bounds, target, side="left"))
        end_t = max(end_t, start_t)
        if r == world - 1:
            end_t = len(traj_first)
        out.append((int(bounds[start_t]), int(bounds[end_t])))
        start_t = end_t
    return out


def shard_queries(queries: Segments, traj_first, rank: int, world: int):
    """This rank's query segments and the offset of its first segment in the full query set."""
    lo, hi = shard_ranges(traj_first, queries.n, world)[rank]
    return queries.take(np.arange(lo, hi)), lo


def merge(parts):
    """Merge per-rank results [(offset, {q_idx, e_idx, t_in, t_out}), ...] into one result in
    global query numbering, sorted by (q_idx, e_idx)."""
    cols = {k: [] for k in ("q_idx", "e_idx", "t_in", "t_out")}
    for off, res in parts:
        cols["q_idx"].append(np.asarray(res["q_idx"], dtype=np.int64) + off)
        for k in ("e_idx", "t_in", "t_out"):
            cols[k].append(np.asarray(res[k]))
    out = {k: (np.concatenate(v) if v else np.zeros(0)) for k, v in cols.items()}
    out["q_idx"] = out["q_idx"].astype(np.uint32)
    out["e_idx"] = out["e_idx"].astype(np.uint32)
    order = np.lexsort((out["e_idx"], out["q_idx"]))
    return {k: v[order] for k, v in out.items()}


def gather_results(local, offset, group=None):
    """All-gather every rank's (offset, result) with torch.distributed (any backend) and merge."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (offset, {k: np.asarray(v) for k, v in local.items()}),
                           group=group)
    return merge(parts)
