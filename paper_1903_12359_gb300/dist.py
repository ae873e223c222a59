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


def sharded_map(ctx, V, F, face_labels):
    """One mesh's pieces shared among the ranks of the current process group.

    Every rank partitions the mesh and solves the DNCP maps of the pieces the
    LPT assignment (on face counts) gives it.  The boundary coordinates go up
    to rank 0 (16 bytes per loop position of an owned piece), which welds them
    and runs the disk map; the welded boundary comes back down (16 bytes per
    loop position); every rank then solves the Laplace problems of its pieces.
    Returns (map [nv, 2] on rank 0, None elsewhere; dict of the bytes each
    exchange moved).  The library does all the arithmetic; this function only
    moves arrays between ranks (object collectives, gloo or NCCL).
    """
    import numpy as np
    import torch.distributed as dist
    ws, rank = dist.get_world_size(), dist.get_rank()
    part = ctx.partition(V, F, face_labels=face_labels)
    try:
        fl, voff, verts, loff, loops = [t.cpu().numpy() for t in part.partition_arrays()]
        K = voff.size - 1
        shards = lpt_shard([float(c) for c in np.bincount(fl, minlength=K)], ws)
        own = np.zeros(K, dtype=bool)
        own[shards[rank]] = True
        part.set_piece_mask(own)
        part.local_param()
        B = part.get_boundary(0).cpu().numpy()
        mine = {i: B[loff[i]:loff[i + 1]] for i in shards[rank]}
        up = [None] * ws if rank == 0 else None
        dist.gather_object(mine, up, dst=0)
        W = [None]
        if rank == 0:
            full = B.copy()
            for d in up:
                for i, b in d.items():
                    full[loff[i]:loff[i + 1]] = b
            part.set_boundary(0, full)
            part.weld()
            W = [part.get_boundary(1).cpu().numpy()]
        dist.broadcast_object_list(W, src=0)
        part.set_boundary(1, W[0])
        out = part.global_solve().cpu().numpy()
        outs = [None] * ws if rank == 0 else None
        dist.gather_object(out, outs, dst=0)
        moved = {"boundary_up_bytes": int(sum(loff[i + 1] - loff[i] for i in range(K)) * 16),
                 "boundary_down_bytes": int(W[0].nbytes)}
        if rank != 0:
            return None, moved
        merged = outs[0].copy()
        for o in outs[1:]:
            take = ~np.isnan(o[:, 0])
            merged[take] = o[take]
        return merged, moved
    finally:
        part.free()
