"""The PCG-schedule autotuner: it picks a valid configuration from its
candidates on a real part, and the pipeline run with the chosen options
matches the FP64 oracle."""
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


@pytest.mark.parametrize("local_precision", [2, 0], ids=["df64", "fp64"])
def test_autotune_picks_a_candidate_and_the_result_is_unchanged(api, local_precision):
    m = meshgen.heightfield_disk_mesh(20000, seed=21, nx=4, ny=2)
    ctx = api.Context(variant=api.DISK, precision=0, tol=1e-12, local_precision=local_precision)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    chosen, ms = ctx.autotune(part, probe_iters=50)
    assert ms > 0
    if local_precision == 2:
        assert chosen["pcg_blocks_per_sm"] in (3, 4) and chosen["pcg_schedule"] in (1, 2, 3, 4)
    else:
        assert chosen["spmv_lanes"] in (1, 2, 4) and chosen["block_rows_log2"] in (8, 9, 10)
    part.local_param()
    part.weld()
    out = part.global_solve().cpu().numpy()
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk").out
    assert np.abs(out - ref).max() < 1e-9
