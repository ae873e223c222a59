"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle.

Partition, boundary loops and CSR pattern: bit-exact.  CSR values: 1e-13
relative (summation order differs).  DNCP coordinates: 1e-9 absolute on the
FP64 path.  Welding on identical inputs: 1e-12 (the kernels repeat the oracle's
operations; reported bitwise when equal).  Final coordinates: 1e-9 (FP64
path), 1e-8 (FP32 solves inside FP64 refinement).  Angle distortion: 1e-6 deg.
"""
import numpy as np
import pytest
import torch

from oracle.mesh import partition as o_partition
from oracle.laplacian import cotan_laplacian
from oracle.dncp import dncp as o_dncp
from oracle.pipeline import pgcp as o_pgcp
from oracle.metrics import angle_distortion
from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _case(name):
    if name == "polar":
        return meshgen.polar_disk_mesh(), "disk"
    if name == "grid4x2":
        return meshgen.heightfield_disk_mesh(3000, seed=3, nx=4, ny=2), "disk"
    if name == "strips8":
        return meshgen.heightfield_disk_mesh(2500, seed=4, nx=8, ny=1), "free"
    if name == "sphere":
        return meshgen.icosphere_sh_mesh(subdiv=3, seed=1), "sphere"
    raise KeyError(name)


CASES = ["polar", "grid4x2", "strips8", "sphere"]
VARIANT = {"free": 0, "disk": 1, "sphere": 2}


def _ctx(api, variant, precision=0, tol=1e-13, **kw):
    return api.Context(variant=VARIANT[variant], precision=precision, tol=tol, **kw)


def _gpu_part(api, m, variant, precision=0, tol=1e-13, **kw):
    ctx = _ctx(api, variant, precision, tol, **kw)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels, closed=(variant == "sphere"))
    return ctx, part


@pytest.mark.parametrize("name", CASES)
def test_partition_and_loops_bit_exact(api, name):
    m, variant = _case(name)
    ctx, part = _gpu_part(api, m, variant)
    fl, voff, verts, loff, loops = [t.cpu().numpy() for t in part.partition_arrays()]
    P = o_partition(m.V, m.F, face_labels=m.face_labels)
    assert part.info()["K"] == P.K
    assert np.array_equal(fl, P.face_label)
    assert np.array_equal(voff, np.concatenate([[0], np.cumsum([v.size for v in P.verts])]))
    assert np.array_equal(verts, np.concatenate(P.verts))
    assert np.array_equal(loff, np.concatenate([[0], np.cumsum([l.size for l in P.loops])]))
    assert np.array_equal(loops, np.concatenate(P.loops))


def test_cut_edge_input_equals_face_labels(api):
    m, _ = _case("grid4x2")
    ctx = _ctx(api, "disk")
    a = ctx.partition(m.V, m.F, cut_edges=m.cut_edges())
    b = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    for x, y in zip(a.partition_arrays(), b.partition_arrays()):
        assert torch.equal(x, y)


@pytest.mark.parametrize("name", CASES)
def test_csr_pattern_bit_exact_values_close(api, name):
    m, variant = _case(name)
    ctx, part = _gpu_part(api, m, variant)
    part.local_param()
    rp, col, val = [t.cpu().numpy() for t in part.csr()]
    P = o_partition(m.V, m.F, face_labels=m.face_labels)
    ptr, cols, vals = [0], [], []
    for i in range(P.K):
        L = cotan_laplacian(m.V[P.verts[i]], P.local_F[i])
        ptr += (L.indptr[1:] + ptr[-1]).tolist()
        cols.append(L.indices)
        vals.append(L.data)
    assert np.array_equal(rp, np.array(ptr))
    assert np.array_equal(col, np.concatenate(cols))
    ref = np.concatenate(vals)
    assert np.abs(val - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("local_precision", [0, 2], ids=["fp64", "df64"])
def test_dncp_matches_direct_solve(api, name, local_precision):
    """FP64 PCG, and double-float PCG inside FP64 refinement: 1e-9 absolute."""
    m, variant = _case(name)
    ctx, part = _gpu_part(api, m, variant, local_precision=local_precision)
    part.local_param()
    assert part.get_stats()["dncp_relres"] <= 1e-13
    u = part.coords(0).cpu().numpy()
    P = o_partition(m.V, m.F, face_labels=m.face_labels)
    voff = np.concatenate([[0], np.cumsum([v.size for v in P.verts])])
    for i in range(P.K):
        ll = np.searchsorted(P.verts[i], P.loops[i])
        ref, _ = o_dncp(m.V[P.verts[i]], P.local_F[i], ll)
        assert np.abs(u[voff[i]:voff[i + 1]] - ref).max() < 1e-9


@pytest.mark.parametrize("name", CASES)
def test_weld_on_identical_inputs(api, name):
    """The welding kernels against the oracle's Algorithms 1-2 (and the disk /
    closed weld) fed with the GPU's own DNCP coordinates."""
    m, variant = _case(name)
    ctx, part = _gpu_part(api, m, variant)
    part.local_param()
    u = part.coords(0).cpu().numpy()
    part.weld()
    w = part.coords(1).cpu().numpy()
    P = o_partition(m.V, m.F, face_labels=m.face_labels)
    voff = np.concatenate([[0], np.cumsum([v.size for v in P.verts])])
    local = [u[voff[i]:voff[i + 1]] for i in range(P.K)]
    r = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant=variant, local=local, map_interior=True)
    worst_b, worst_i, scale = 0.0, 0.0, 0.0
    for i in range(P.K):
        g = w[voff[i]:voff[i + 1]]
        o = r.welded[i]
        on = np.zeros(g.size, dtype=bool)
        on[np.searchsorted(P.verts[i], P.loops[i])] = True
        worst_b = max(worst_b, np.abs(g[on] - o[on]).max())
        worst_i = max(worst_i, np.abs(g[~on] - o[~on]).max() if (~on).any() else 0.0)
        scale = max(scale, np.abs(o[on]).max())
    assert worst_b <= 1e-12 * max(scale, 1.0)       # FP64 boundary: same operations
    assert worst_i <= 2e-3 * max(scale, 1.0)        # FP32 interior weld map (warm start)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision,local_precision,tol", [(0, 0, 1e-9), (1, 0, 1e-8), (2, 2, 1e-9), (1, 2, 1e-8)],
                         ids=["fp64", "fp32ref", "df64", "df64+fp32ref"])
def test_final_coordinates_match_oracle(api, name, precision, local_precision, tol):
    m, variant = _case(name)
    ctx, part = _gpu_part(api, m, variant, precision=precision, tol=1e-13, local_precision=local_precision)
    part.local_param()
    part.weld()
    out = part.global_solve().cpu().numpy()
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant=variant).out
    assert np.abs(out - ref).max() < tol
    st = part.stats
    assert st["final_relres"] <= 1e-13 and st["seam_mismatch"] < 1e-12
    met = part.metrics(torch.as_tensor(out, device="cuda"))
    ad = angle_distortion(m.V, m.F, ref)
    for k in ("mean", "max", "median", "iqr", "sd"):
        assert abs(met[k] - ad[k]) < 1e-6, k
    assert met["flips"] == 0


def test_metrics_kernel_on_a_fixed_input(api):
    m, _ = _case("grid4x2")
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk").out
    ctx, part = _gpu_part(api, m, "disk")
    met = part.metrics(torch.as_tensor(ref, device="cuda"))
    ad = angle_distortion(m.V, m.F, ref)
    for k in ("mean", "sd", "median", "iqr", "max"):
        assert abs(met[k] - ad[k]) < 1e-9, k
    assert met["n_corners"] == 3 * m.nf


def test_errors_are_status_codes(api):
    m = meshgen.polar_disk_mesh(rings=4, sectors=8)
    ctx = _ctx(api, "disk")
    with pytest.raises(api.PgcpError) as e:
        ctx.partition(m.V, m.F, cut_edges=np.array([[0, 20]]))
    assert e.value.code == "ARG"
    lab = np.zeros(m.nf, dtype=np.int32)
    lab[:8] = 1
    with pytest.raises(api.PgcpError) as e:
        ctx.partition(m.V, m.F, face_labels=lab)
    assert e.value.code == "TOPOLOGY"
    F = np.concatenate([m.F, [[0, 1, 2]]])
    with pytest.raises(api.PgcpError) as e:
        ctx.partition(m.V, F, face_labels=np.zeros(F.shape[0], dtype=np.int32))
    assert e.value.code in ("NONMANIFOLD", "ARG")
    # the context stays usable
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    assert part.info()["K"] == 2


def test_batch_equals_single_meshes(api):
    ms = [meshgen.heightfield_disk_mesh(1500 + 500 * i, seed=10 + i, nx=2 + i, ny=2) for i in range(3)]
    ctx = _ctx(api, "disk")
    part = ctx.partition_batch([(m.V, m.F, m.face_labels) for m in ms])
    part.local_param()
    part.weld()
    out = part.global_solve().cpu().numpy()
    off = 0
    for m in ms:
        p1 = ctx.partition(m.V, m.F, face_labels=m.face_labels)
        p1.local_param()
        p1.weld()
        o1 = p1.global_solve().cpu().numpy()
        assert np.abs(out[off:off + m.nv] - o1).max() < 1e-10
        off += m.nv


def test_one_shot_host_io(api):
    m, _ = _case("polar")
    ctx = _ctx(api, "disk", precision=1, tol=1e-12)
    out_h, st = ctx.run(m.V, m.F, face_labels=m.face_labels, host=True)
    out_d, _ = ctx.run(m.V, m.F, face_labels=m.face_labels, host=False)
    assert isinstance(out_h, np.ndarray) and out_h.shape == (m.nv, 2)
    assert np.abs(out_h - out_d.cpu().numpy()).max() < 1e-10
    assert st["final_relres"] <= 1e-12


@pytest.mark.slow
def test_partition_full_size_bit_exact(api):
    """The 1M-vertex workload: partition, vertex lists and loops bit-exact."""
    m = meshgen.heightfield_disk_mesh(1_000_000, seed=0, nx=4, ny=2)
    ctx = _ctx(api, "disk")
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    fl, voff, verts, loff, loops = [t.cpu().numpy() for t in part.partition_arrays()]
    P = o_partition(m.V, m.F, face_labels=m.face_labels)
    assert np.array_equal(fl, P.face_label)
    assert np.array_equal(verts, np.concatenate(P.verts))
    assert np.array_equal(loops, np.concatenate(P.loops))


@pytest.mark.parametrize("schedule", [1, 2, 3, 4], ids=["static", "dynamic", "roundrobin", "onereduction"])
@pytest.mark.parametrize("name", ["grid4x2", "sphere"])
def test_dncp_and_final_under_every_pcg_schedule(api, name, schedule):
    """The three work schedules of the mixed-precision PCG give the oracle's map."""
    m, variant = _case(name)
    ctx, part = _gpu_part(api, m, variant, precision=1, tol=1e-13, local_precision=2, pcg_schedule=schedule)
    part.local_param()
    u = part.coords(0).cpu().numpy()
    P = o_partition(m.V, m.F, face_labels=m.face_labels)
    voff = np.concatenate([[0], np.cumsum([v.size for v in P.verts])])
    for i in range(P.K):
        ll = np.searchsorted(P.verts[i], P.loops[i])
        ref, _ = o_dncp(m.V[P.verts[i]], P.local_F[i], ll)
        assert np.abs(u[voff[i]:voff[i + 1]] - ref).max() < 1e-9
    part.weld()
    out = part.global_solve().cpu().numpy()
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant=variant).out
    assert np.abs(out - ref).max() < 1e-8
