"""The library at the full sizes of the three workloads, checked by what the
oracle can compute at that size:
- per-piece FP64 residuals with the oracle's own cotangent Laplacian;
- the welding on identical inputs against the oracle's Algorithms 1-2 and
  disk map (boundary values);
- no flipped triangles, the boundary on the unit circle or every point on
  the unit sphere, and seams that agree;
- for the uneven batch, the meshes that fail alone are status codes; the whole
  batch, those meshes included, runs in one call with them dropped (NaN), the
  others equal the meshes run one by one, and the smallest meshes equal the
  oracle.
"""
import numpy as np
import pytest
import torch

from oracle.laplacian import cotan_laplacian
from oracle.metrics import fold_check
from oracle.pipeline import pgcp as o_pgcp
from paper_1903_12359_gb300 import meshgen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _pieces(part):
    fl, voff, verts, loff, loops = [t.cpu().numpy() for t in part.partition_arrays()]
    out = []
    for i in range(voff.size - 1):
        v = verts[voff[i]:voff[i + 1]]
        ll = np.searchsorted(v, loops[loff[i]:loff[i + 1]])
        out.append((voff[i], voff[i + 1], v, ll, fl))
    return out


def _piece_faces(F, fl, i, v):
    f = F[fl == i]
    return np.searchsorted(v, f)


def _final_residuals(m, part, final):
    """max over pieces and coordinates of ||L_II u_I + L_IB u_B|| / ||L_IB u_B||."""
    worst = 0.0
    fl = part.partition_arrays()[0].cpu().numpy()
    for i, (a, b, v, ll, _) in enumerate(_pieces(part)):
        L = cotan_laplacian(m.V[v], _piece_faces(m.F, fl, i, v))
        u = final[a:b]
        isb = np.zeros(b - a, dtype=bool)
        isb[ll] = True
        inner = ~isb
        for c in (u.real, u.imag):
            r = L[inner] @ c
            rb = L[inner][:, isb] @ c[isb]
            worst = max(worst, np.linalg.norm(r) / np.linalg.norm(rb))
    return worst


def test_disk_1m_full_size(api):
    m = meshgen.heightfield_disk_mesh(1_000_000, seed=0, nx=4, ny=2)
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-10, local_precision=api.DF64_REFINED)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels)
    part.local_param()
    u_local = part.coords(0).cpu().numpy()
    part.weld()
    welded = part.coords(1).cpu().numpy()
    out = part.global_solve().cpu().numpy()
    st = part.stats
    assert st["final_relres"] <= 1e-10 and st["dncp_relres"] <= 1e-10 and st["seam_mismatch"] < 1e-9
    final = part.coords(2).cpu().numpy()
    assert _final_residuals(m, part, final) <= 1e-10
    # mesh boundary on the unit circle, no flipped triangle
    r = np.hypot(out[:, 0], out[:, 1])
    assert np.abs(r[np.isclose(np.hypot(m.V[:, 0], m.V[:, 1]), 1.0)] - 1.0).max() < 1e-12
    assert fold_check(m.V, m.F, out)["flips"] == 0
    # welding (and disk map) on identical inputs: boundary values against the oracle
    pcs = _pieces(part)
    local = [u_local[a:b] for a, b, *_ in pcs]
    ref = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk", local=local)
    scale = 1.0
    for i, (a, b, v, ll, _) in enumerate(pcs):
        d = np.abs(welded[a:b][ll] - ref.welded[i][ll]).max()
        assert d <= 1e-11 * scale, (i, d)


def test_sphere_655k_full_size(api):
    m = meshgen.icosphere_sh_mesh(subdiv=8, seed=0)
    ctx = api.Context(variant=api.SPHERE, precision=api.FP32_REFINED, tol=1e-10, local_precision=api.DF64_REFINED)
    part = ctx.partition(m.V, m.F, face_labels=m.face_labels, closed=True)
    part.local_param()
    part.weld()
    out = part.global_solve().cpu().numpy()
    st = part.stats
    assert m.nv == 655362 and st["K"] == 8
    assert st["final_relres"] <= 1e-10 and st["seam_mismatch"] < 1e-9
    assert np.abs(np.linalg.norm(out, axis=1) - 1.0).max() < 1e-12
    assert _final_residuals(m, part, part.coords(2).cpu().numpy()) <= 1e-10
    met = part.metrics(torch.as_tensor(out, device="cuda"))
    assert met["flips"] == 0 and met["n_corners"] == 3 * m.nf


def test_uneven_batch_full_size(api):
    ms = meshgen.uneven_batch(n_mesh=256, seed=0)
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-10, local_precision=api.DF64_REFINED)
    good, rejected = [], []
    for i, x in enumerate(ms):
        try:
            p = ctx.partition(x.V, x.F, face_labels=x.face_labels)
            p.local_param()
            p.weld()
            p.global_solve()
            good.append(i)
        except api.PgcpError as e:           # a status code, never a crash
            assert e.code in ("NUMERIC", "NO_CONVERGENCE", "SCHEDULE")
            rejected.append((i, e.code))
    assert len(good) >= 0.9 * len(ms), rejected
    # the whole batch, the meshes that fail alone included, in one call
    part = ctx.partition_batch([(x.V, x.F, x.face_labels) for x in ms])
    part.local_param()
    part.weld()
    out = part.global_solve().cpu().numpy()
    assert part.stats["final_relres"] <= 1e-10 and part.stats["dncp_relres"] <= 1e-10
    offs = np.concatenate([[0], np.cumsum([x.nv for x in ms])])
    # a mesh that fails alone is dropped (NaN output); a mesh at the edge of the
    # FP64 welding domain may also be dropped (its DNCP map differs at the 1e-10
    # level in the batch); the others go on
    status = part.mesh_status()
    dropped = [j for j, c in enumerate(status) if c != "OK"]
    assert len(dropped) <= len(rejected) + 0.05 * len(ms), (dropped, rejected)
    for j in dropped:
        assert status[j] == "NUMERIC" and np.isnan(out[offs[j]:offs[j + 1]]).all()
    kept = [j for j in range(len(ms)) if j not in dropped]
    assert np.isfinite(out[np.concatenate([np.arange(offs[j], offs[j + 1]) for j in kept])]).all()
    # batch = meshes one by one, on a sample
    both = [j for j in kept if j in good]
    for j in both[::max(1, len(both) // 6)][:6]:
        x = ms[j]
        p = ctx.partition(x.V, x.F, face_labels=x.face_labels)
        p.local_param()
        p.weld()
        o1 = p.global_solve().cpu().numpy()
        assert np.abs(out[offs[j]:offs[j + 1]] - o1).max() < 1e-8
    # the smallest meshes against the oracle
    for j in sorted(both, key=lambda t: ms[t].nv)[:3]:
        x = ms[j]
        ref = o_pgcp(x.V, x.F, face_labels=x.face_labels, variant="disk").out
        assert np.abs(out[offs[j]:offs[j + 1]] - ref).max() < 1e-8
