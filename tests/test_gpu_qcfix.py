"""The fold-over fix (Section 4.5, Algorithm 3's last step; composition,
Section 3.5) through the C ABI against the oracle's fix (oracle/qcfix.py) on
host-made folding inputs: the same fold counts and rounds, coordinates within
1e-8, no folded face and |mu| < 1 afterwards, boundary values untouched; a map
that does not fold is returned bit for bit; closed parts are refused."""
import numpy as np
import pytest
import torch

import oracle.qcfix as Q
from oracle.laplacian import cotan_laplacian
from oracle.mesh import partition
from oracle.metrics import fold_check
from oracle.pipeline import harmonic_solve, pgcp
from paper_1903_12359_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api as a
    return a


def _dragged(V, F, loop, w):
    z = V[:, 0] + 1j * V[:, 1]
    isb = np.zeros(len(V), dtype=bool)
    isb[loop] = True
    inner = np.nonzero(~isb)[0]
    c = inner[np.argmin(np.abs(z[inner] - 0.2))]
    ring = np.unique(F[(F == c).any(axis=1)].ravel())
    ring = ring[ring != c]
    wf = w.copy()
    wf[c] = w[c] + 3.0 * np.abs(w[ring] - w[c]).max()
    return wf


def _gpu_fix(api, V, F, labels, U):
    ctx = api.Context(variant=api.DISK, precision=api.FP32_REFINED, tol=1e-13)
    part = ctx.partition(V, F, face_labels=labels)
    Ud = torch.tensor(U, device="cuda")
    rep = part.fix_folds(Ud)
    return Ud.cpu().numpy(), rep


def _check_against_oracle(api, V, F, labels, U):
    P = partition(V, F, face_labels=labels)
    ref, counts = Q.fix_folds(V, F, P, U)
    got, rep = _gpu_fix(api, V, F, labels, U)
    assert rep["folded_before"] == sum(c[0] for c in counts)
    assert rep["rounds"] == max(c[1] for c in counts)
    assert rep["folded_after"] == 0 and all(c[2] == 0 for c in counts)
    assert np.abs(got - ref).max() < 1e-8, np.abs(got - ref).max()
    fc = fold_check(V, F, got)
    assert fc["flips"] == 0 and fc["max_mu"] < 1.0
    for i in range(P.K):   # boundary values kept
        b = P.loops[i]
        assert np.array_equal(got[b], U[b])
    return rep


def test_dragged_vertex_in_one_piece(api):
    m = meshgen.heightfield_disk_mesh(3000, seed=3, nx=2, ny=1)
    res = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk")
    P = res.part
    U = res.out.copy()
    g1 = P.verts[1]
    loop1 = np.searchsorted(g1, P.loops[1])
    w1 = U[g1, 0] + 1j * U[g1, 1]
    wf = _dragged(m.V[g1], P.local_F[1], loop1, w1)
    k = np.nonzero(wf != w1)[0][0]
    U[g1[k]] = [wf[k].real, wf[k].imag]
    rep = _check_against_oracle(api, m.V, m.F, m.face_labels, U)
    assert rep["pieces_fixed"] == 1


def test_fold_next_to_a_concave_boundary(api):
    m = meshgen.polar_disk_mesh(rings=12, sectors=24, jitter=0.0)
    V = m.V.copy()
    V[:, 2] = 0.0
    labels = np.zeros(m.F.shape[0], dtype=np.int32)
    loop = partition(V, m.F, face_labels=labels).loops[0]
    th = np.angle(V[loop, 0] + 1j * V[loop, 1])
    wb = (1.0 + 0.6 * np.cos(5 * th)) * np.exp(1j * th)
    w = harmonic_solve(cotan_laplacian(V, m.F), loop, wb)
    U = np.stack([w.real, w.imag], axis=1)
    rep = _check_against_oracle(api, V, m.F, labels, U)
    assert rep["rounds"] >= 2


def test_map_without_folds_is_unchanged_and_closed_parts_are_refused(api):
    m = meshgen.heightfield_disk_mesh(3000, seed=3, nx=4, ny=2)
    U = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk").out
    got, rep = _gpu_fix(api, m.V, m.F, m.face_labels, U)
    assert rep == {"folded_before": 0, "folded_after": 0, "rounds": 0, "pieces_fixed": 0}
    assert np.array_equal(got, U)
    s = meshgen.icosphere_sh_mesh(subdiv=2, seed=0)
    ctx = api.Context(variant=api.SPHERE)
    part = ctx.partition(s.V, s.F, face_labels=s.face_labels, closed=True)
    with pytest.raises(api.PgcpError) as e:   # the library refuses closed parts
        part.fix_folds(torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda"))
    assert e.value.code == "ARG"
