"""The one-call forms (pgcp_free_boundary, pgcp_disk, pgcp_sphere,
pgcp_batch_run) equal the step-by-step calls on the same inputs, and the FP64
oracle within the parity tolerance."""
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


@pytest.mark.parametrize("variant", ["free", "disk", "sphere"])
def test_one_call_forms_match_the_oracle(api, variant):
    if variant == "sphere":
        m = meshgen.icosphere_sh_mesh(subdiv=3, seed=1)
    elif variant == "free":
        m = meshgen.heightfield_disk_mesh(2500, seed=4, nx=8, ny=1)
    else:
        m = meshgen.heightfield_disk_mesh(3000, seed=3, nx=4, ny=2)
    ctx = api.Context(variant=api.FREE, precision=0, tol=1e-13)   # the call sets its own variant
    out, st = api.one_call(ctx, variant, m.V, m.F, face_labels=m.face_labels)
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant=variant).out
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-9
    assert st["final_relres"] <= 1e-13
    assert ctx.options.variant == api.FREE


def test_batch_run_equals_single_meshes(api):
    ms = [meshgen.heightfield_disk_mesh(1500 + 700 * i, seed=30 + i, nx=2 + i, ny=2) for i in range(3)]
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-11)
    outs, status, st = api.batch_run(ctx, [(m.V, m.F, m.face_labels) for m in ms])
    assert status == ["OK"] * 3 and st["K"] == sum(int(m.face_labels.max()) + 1 for m in ms)
    for m, o in zip(ms, outs):
        single, _ = api.one_call(ctx, "disk", m.V, m.F, face_labels=m.face_labels)
        assert np.abs(o.cpu().numpy() - single.cpu().numpy()).max() < 1e-9
