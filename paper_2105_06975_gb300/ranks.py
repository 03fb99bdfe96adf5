"""Multi-rank host logic: one process per GPU, independent windows.

Assimilation windows are independent saddle-point problems, so the path
shards with no data-path collective: each rank solves its own windows and the
only communication is the timing reduction (max over ranks) and the count of
solved windows.  Everything here is host logic over torch.distributed and runs
with the gloo backend on CPU as well as with NCCL on GPUs.
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def dist_info() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def window_seed(master_seed: int, rank: int) -> int:
    """Seed of the window rank `rank` solves in the one-window-per-rank runs
    (window w of master seed m draws with 1000 m + w)."""
    return 1000 * int(master_seed) + int(rank)


def partition_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Assign window indices to ranks, largest first to the least loaded rank
    (longest-processing-time rule; ties go to the lowest rank).  Every index
    appears exactly once; the result is the same on every rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return parts


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the job's wall time is the slowest
    rank's); the identity without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_this_rank: float, ms_this_rank: float, device=None) -> Tuple[float, float]:
    """(units per second over the whole job, max milliseconds over ranks):
    all ranks' units divided by the slowest rank's time."""
    ms = max_over_ranks(ms_this_rank, device)
    units = sum_over_ranks(units_this_rank, device)
    return (units * 1e3 / ms if ms > 0 else 0.0), ms
