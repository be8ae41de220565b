"""Multi-GPU: independent replicas (one process per GPU, no data-path
collective).

A single hull is not split across GPUs here; batched point sets and serving
requests shard by set or request with no exchange at all, and the bench runs
one replica of its workload per rank (weak scaling).  This module holds the
host-side pieces: the rank environment, the contiguous split of items over
ranks, and the max-over-ranks timing that makes the whole-job rate.
"""
from __future__ import annotations

import os


def dist_env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_range(n_items: int, rank: int, ws: int):
    """Contiguous share [lo, hi) of n_items for rank `rank` of `ws`; the
    shares of all ranks partition [0, n_items) and differ by at most one."""
    if ws < 1 or not 0 <= rank < ws:
        raise ValueError("rank outside the world")
    lo = n_items * rank // ws
    hi = n_items * (rank + 1) // ws
    return lo, hi


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (the job ends when its slowest rank
    does); the value itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    if seconds_max <= 0:
        raise ValueError("non-positive time")
    return units_per_rank * ws / seconds_max
