"""Multi-process plumbing of the weak-scaling runs (one process per GPU).

The hot path shards by independent problems: each rank owns whole meshes (or
whole pieces) and runs the library on them alone; no collective sits on the
data path.  Ranks meet only to time a step (barrier, maximum of the per-rank
times) and to total the work.
"""
from __future__ import annotations

import os


def env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def lpt_shard(costs, world_size: int):
    """Longest-processing-time-first assignment of items (e.g. meshes by their
    stored entries) to ranks: items in decreasing cost, each to the least
    loaded rank (ties: lower rank, then lower item index).  Returns per-rank
    lists of item indices, each in increasing order."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world_size
    out = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def _reduce(x: float, op_name: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "MAX", device)


def sum_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "SUM", device)


def throughput(units_per_rank: float, ms_per_rank: float, device=None) -> float:
    """Whole-job rate: all ranks' units over the slowest rank's time."""
    units = sum_over_ranks(units_per_rank, device)
    ms = max_over_ranks(ms_per_rank, device)
    return units / (ms / 1000.0)
