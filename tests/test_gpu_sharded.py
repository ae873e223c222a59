"""The sharded-pieces path of the library (paper_1903_12359_gb300.dist
.sharded_map): two ranks (gloo, both on cuda:0, separate processes) each solve
the DNCP and Laplace problems of their pieces, exchanging only boundary
coordinates through rank 0's welds.  The merged map equals the single-process
library run (cold-started final solve) to the solve's accuracy, every vertex
is written by exactly one rank, and the exchanged bytes are the boundaries'."""
import os
import socket

import numpy as np
import pytest

from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    from paper_1903_12359_gb300 import api, dist as pd
    m = meshgen.heightfield_disk_mesh(20000, seed=7, nx=4, ny=2)
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-13, warm_start=api.WARM_COLD)
    out, moved = pd.sharded_map(ctx, m.V, m.F, m.face_labels)
    if rank == 0:
        np.save(out_path, out)
        np.save(out_path + ".moved.npy", np.array([moved["boundary_up_bytes"], moved["boundary_down_bytes"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_match_the_single_process_run(tmp_path):
    from paper_1903_12359_gb300 import build
    build.build()
    import torch.multiprocessing as mp
    out_path = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out_path), nprocs=2, start_method="spawn")
    merged = np.load(out_path)
    up, down = np.load(out_path + ".moved.npy")
    from paper_1903_12359_gb300 import api
    m = meshgen.heightfield_disk_mesh(20000, seed=7, nx=4, ny=2)
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-13, warm_start=api.WARM_COLD)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    part.local_param()
    part.weld()
    ref = part.global_solve().cpu().numpy()
    n_loop = part.info()["n_loop"]
    assert not np.isnan(merged).any()
    assert np.abs(merged - ref).max() < 1e-9, np.abs(merged - ref).max()
    assert up == down == 16 * n_loop
