"""Static-schedule solves run in launches of 256 iterations. Between launches
the runs are rebuilt over the pieces that have not converged. A batch of one
large mesh and several small ones (the small pieces converge in the first
launch, the large ones need several) must give the same maps as the meshes
solved one by one and as deterministic mode, which keeps one launch and the
original runs, and the FP64 oracle on a small mesh."""
import numpy as np
import pytest

from oracle.pipeline import pgcp as o_pgcp
from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def test_rebuilt_runs_give_the_same_maps(api):
    big = meshgen.heightfield_disk_mesh(150_000, seed=21, nx=2, ny=2)
    small = [meshgen.heightfield_disk_mesh(2500 + 500 * i, seed=22 + i, nx=2, ny=2) for i in range(4)]
    ms = [big] + small
    outs = {}
    stats = {}
    for det in (0, 1):
        ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-11, deterministic=det)
        part = ctx.partition_batch([(m.V, m.F, m.face_labels) for m in ms])
        part.local_param()
        st_local = part.get_stats()
        part.weld()
        out = part.global_solve().cpu().numpy()
        assert part.mesh_status() == ["OK"] * len(ms)
        outs[det] = out
        stats[det] = (st_local, dict(part.stats))
        part.free()
    st_local, st = stats[0]
    # the large pieces outlive the first launch of each refinement step
    assert st_local["dncp_iters"] > 4 * 256 and st_local["pcg_launches"] >= 6
    assert st["dncp_relres"] <= 1e-11 and st["final_relres"] <= 1e-11
    assert np.abs(outs[0] - outs[1]).max() < 1e-8
    offs = np.concatenate([[0], np.cumsum([m.nv for m in ms])])
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-11)
    for j, m in enumerate(ms):
        single, _ = api.one_call(ctx, "disk", m.V, m.F, face_labels=m.face_labels)
        assert np.abs(outs[0][offs[j]:offs[j + 1]] - single.cpu().numpy()).max() < 1e-8
    ref = o_pgcp(small[0].V, small[0].F, face_labels=small[0].face_labels, variant="disk").out
    assert np.abs(outs[0][offs[1]:offs[2]] - ref).max() < 1e-8
