"""Parity at the benchmarked configuration: the 1M-vertex height-field disk
(seed 0, 4 x 2 cut grid, 8 pieces) with the bench's solver options, against
the FP64 oracle run on the same mesh.

Two stopping tolerances (relative residual per piece and coordinate, the
reading of Section 4.5 "solve the Laplace equation"):
- 1e-10, the residual the headline metric names;
- 1e-12, the bench's stopping rule.
(At 1e-13 the double-float DNCP refinement of the 1M mesh stops just above
the tolerance; the smaller parity cases run at 1e-13.)

For each, the DNCP map of every piece (Section 4.2), the final disk map and the
angle-distortion statistics (Section 5) are compared element by element, and
the measured maximum errors are printed (and appended as one JSON line to the
file named by PGCP_PARITY_REPORT, when set).

Bars: a relative residual bounds the coordinate error only through the
conditioning of the piece systems.  At 1e-10 the final map meets the
mixed-precision bar of 1e-8 and the mean, sd, median and IQR of |d| agree to
1e-6 degrees, but the max of |d| -- one corner of a triangle about 2e-3 wide --
moves by about 1e-5 degrees; that is why the bench stops at 1e-12, where every
statistic must agree to 1e-6 degrees.  The DNCP map is an intermediate whose
error is cond(A~) * relres * |u| at worst: the scaled DNCP systems have
cond 6e7-1e8 already on 10k-row pieces (113k rows here), a worst case above
6e-5 at 1e-12; its bar is 1e-7.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle.metrics import angle_distortion
from oracle.pipeline import pgcp as o_pgcp
from paper_1903_12359_gb300 import meshgen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def bench_case():
    m = meshgen.heightfield_disk_mesh(1_000_000, seed=0, nx=4, ny=2)
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk", workers=min(8, max(1, cores)))
    return m, ref, angle_distortion(m.V, m.F, ref.out)


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
def test_bench_mesh_matches_oracle(api, bench_case, tol):
    m, ref, ad = bench_case
    ctx = api.Context(variant=api.DISK, precision=api.DF64_REFINED, tol=tol, local_precision=api.DF64_REFINED,
                      warm_start=api.WARM_COLD)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    part.local_param()
    local = part.coords(0).cpu().numpy()
    part.weld()
    out = part.global_solve()
    st = part.stats
    assert st["dncp_relres"] <= tol and st["final_relres"] <= tol
    _, voff, *_ = part.partition_arrays()
    voff = voff.cpu().numpy()
    assert voff.size - 1 == ref.part.K == 8
    dncp_err = max(float(np.abs(local[voff[i]:voff[i + 1]] - ref.local[i]).max()) for i in range(ref.part.K))
    outh = out.cpu().numpy()
    final_err = float(np.abs(outh - ref.out).max())
    met = part.metrics(out)
    d_err = {k: abs(met[k] - ad[k]) for k in ("mean", "sd", "median", "iqr", "max")}
    report = {"tol": tol, "dncp_max_abs_err": dncp_err, "final_max_abs_err": final_err,
              "abs_d_stat_err_deg": d_err, "dncp_iters": st["dncp_iters"], "final_iters": st["final_iters"],
              "dncp_relres": st["dncp_relres"], "final_relres": st["final_relres"]}
    print("bench-config parity", json.dumps(report))
    if os.environ.get("PGCP_PARITY_REPORT"):
        with open(os.environ["PGCP_PARITY_REPORT"], "a") as f:
            f.write(json.dumps(report) + "\n")
    assert final_err < 1e-8, report
    assert max(d_err[k] for k in ("mean", "sd", "median", "iqr")) < 1e-6, report
    assert d_err["max"] < (1e-4 if tol > 1e-12 else 1e-6), report
    assert met["flips"] == 0
    if tol <= 1e-12:
        assert dncp_err < 1e-7, report
