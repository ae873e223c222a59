"""The multi-rank plumbing of the weak-scaling bench on CPU: two gloo ranks
(127.0.0.1) reduce their step times and work exactly as the GPU ranks do, and
the longest-processing-time sharding covers every item once."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1903_12359_gb300 import dist as pd


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(WORLD_SIZE=str(ws), RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        w, r, l = pd.env()
        ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
        units = 1_000_000.0 * (rank + 1)
        q.put((r, w, pd.max_over_ranks(ms), pd.sum_over_ranks(units), pd.throughput(units, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, mx, tot, rate in res:
        assert w == 2 and mx == 150.0 and tot == 3_000_000.0
        assert rate == pytest.approx(3_000_000.0 / 0.150)


def test_lpt_shard_covers_every_item_once_and_balances():
    costs = [int(c) for c in (97, 12, 55, 55, 3, 80, 41, 41, 7, 66, 20, 90)]
    for ws in (1, 2, 3, 4, 8):
        parts = pd.lpt_shard(costs, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # Graham's bound for LPT: at most 4/3 of the optimum, which is >= the mean and the largest item
        assert max(loads) <= 4.0 / 3.0 * max(sum(costs) / ws, max(costs)) + 1e-9
    assert pd.lpt_shard([5, 5], 2) == [[0], [1]]
