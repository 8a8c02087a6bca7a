"""Replica execution over ranks (one process per GPU).

The assimilation path has no exchange step: sweep members, ensemble
realisations and served jobs are independent.  Ranks therefore only share
a start barrier and the timing reduction; work is split by member index.
"""
from __future__ import annotations

import os


def env_world():
    """(rank, local_rank, world_size) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(count: int, rank: int, world: int):
    """Contiguous block [start, stop) of `count` members owned by `rank`;
    blocks differ in size by at most one and cover every member once."""
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (1 rank: the value itself)."""
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


def whole_job_rate(units_per_rank: float, seconds_per_rank: float, device=None) -> float:
    """Units of all ranks divided by the slowest rank's time."""
    return sum_over_ranks(units_per_rank, device) / max_over_ranks(seconds_per_rank, device)
