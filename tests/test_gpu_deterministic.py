"""Deterministic mode (pgcp_options.deterministic = 1): the reductions that steer
the solves are summed in a fixed order, so two runs on the same inputs give
bitwise identical maps and iteration counts; the maps still equal the FP64
oracle within the parity tolerance.  Covered: the double-float DNCP and FP32
final solves with their FP64 refinement, the learned warm start, a batch of
meshes, the autotuner's candidate list, and the FP64 solver's refusal."""
import os

import numpy as np
import pytest

from oracle.pipeline import pgcp as o_pgcp
from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _run(api, m, warm=None, gnn_path=None, **kw):
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, local_precision=api.DF64_REFINED,
                      tol=1e-11, deterministic=1, warm_start=api.WARM_WELDMAP if warm is None else warm, **kw)
    if gnn_path:
        ctx.set_gnn(api.Gnn(ctx, path=gnn_path))
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    part.local_param()
    part.weld()
    out = part.global_solve().cpu().numpy()
    st = dict(part.stats)
    part.free()
    return out, st


KEYS = ("dncp_iters", "final_iters", "dncp_refine", "final_refine", "dncp_relres", "final_relres", "learned_pieces")


def test_two_runs_are_bitwise_identical_and_match_the_oracle(api):
    m = meshgen.heightfield_disk_mesh(40_000, seed=11, nx=4, ny=2)
    a, sa = _run(api, m)
    b, sb = _run(api, m)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    assert all(sa[k] == sb[k] for k in KEYS), {k: (sa[k], sb[k]) for k in KEYS}
    assert sa["dncp_relres"] <= 1e-11 and sa["final_relres"] <= 1e-11
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk").out
    assert np.abs(a - ref).max() < 1e-8


def test_learned_start_is_deterministic(api):
    m = meshgen.heightfield_disk_mesh(30_000, seed=12, nx=4, ny=2)
    w = os.path.join(ROOT, "paper_1903_12359_gb300", "weights", "mpnn_disk.bin")
    a, sa = _run(api, m, warm=api.WARM_LEARNED, gnn_path=w)
    b, sb = _run(api, m, warm=api.WARM_LEARNED, gnn_path=w)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    assert all(sa[k] == sb[k] for k in KEYS), {k: (sa[k], sb[k]) for k in KEYS}
    c, _ = _run(api, m)                       # the weld-map start reaches the same map
    assert np.abs(a - c).max() < 1e-8


def test_batch_is_deterministic(api):
    ms = [meshgen.heightfield_disk_mesh(4000 + 3000 * i, seed=40 + i, nx=2 + i, ny=2) for i in range(3)]
    outs = []
    for _ in range(2):
        ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-11, deterministic=1)
        o, status, st = api.batch_run(ctx, [(m.V, m.F, m.face_labels) for m in ms])
        assert status == ["OK"] * 3
        outs.append(([x.cpu().numpy() for x in o], st))
    for x, y in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(x.view(np.uint64), y.view(np.uint64))
    assert outs[0][1]["dncp_iters"] == outs[1][1]["dncp_iters"]


def test_autotune_keeps_the_static_schedule(api):
    m = meshgen.heightfield_disk_mesh(20_000, seed=13, nx=4, ny=2)
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-10, deterministic=1)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    chosen, _ = ctx.autotune(part, probe_iters=50)
    assert chosen["pcg_schedule"] == 1 and chosen["pcg_blocks_per_sm"] in (3, 4)


def test_fp64_solver_refuses_deterministic_mode(api):
    m = meshgen.heightfield_disk_mesh(3000, seed=14, nx=2, ny=2)
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, local_precision=api.FP64, deterministic=1)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    with pytest.raises(api.PgcpError) as e:
        part.local_param()
    assert e.value.code == "ARG"
