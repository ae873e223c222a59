"""Pins of the oracle's fold-over fix (oracle/qcfix.py; Section 4.5 and
Algorithm 3's last step, Beltrami coefficient and composition, Section 3.5).

- The Beltrami coefficient of an affine map z + b conj(z) is b in the plane's
  frame, so b exp(-2 i theta) in a face frame rotated by theta (closed form).
- The linear Beltrami solver with nu = 0 is the cotangent Laplacian.
- The solver reproduces a non-conformal map from its own coefficients and
  boundary values (the exactness of the linear-element discretisation).
- Two host-made folds -- an interior vertex dragged across its ring, and the
  harmonic map onto a star-shaped boundary -- are removed: no face folds and
  |mu| < 1 after the fix, with the boundary values untouched.
- A map that does not fold is returned unchanged.
"""
import numpy as np
import pytest

import oracle.qcfix as Q
from oracle.laplacian import cotan_laplacian
from oracle.mesh import partition
from oracle.pipeline import harmonic_solve, pgcp
from paper_1903_12359_gb300 import meshgen


def _single_piece(N=3000, seed=3):
    m = meshgen.heightfield_disk_mesh(N, seed=seed, nx=1, ny=1)
    P = partition(m.V, m.F, face_labels=m.face_labels)
    assert P.K == 1
    g = P.verts[0]
    return m, m.V[g], P.local_F[0], np.searchsorted(g, P.loops[0])


def _dragged(V, F, loop, w):
    """Move one interior vertex 3 ring-radii across its ring."""
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


def test_affine_map_coefficient_is_closed_form():
    m = meshgen.polar_disk_mesh(rings=8, sectors=16)
    V = m.V.copy()
    V[:, 2] = 0.0
    z = V[:, 0] + 1j * V[:, 1]
    # each face's frame has p0 -> p1 on its +x axis: the plane rotated by theta
    e = z[m.F[:, 1]] - z[m.F[:, 0]]
    rot = np.exp(-2j * np.angle(e))
    for b in (0.3 - 0.2j, -0.5j, 0.0):
        mu = Q.beltrami(V, m.F, 2.0 * z + b * 2.0 * np.conj(z) + 1.0)
        assert np.abs(mu - b * rot).max() < 1e-13
        assert np.abs(np.abs(mu) - abs(b)).max() < 1e-13


def test_solver_with_zero_coefficient_is_the_cotan_laplacian():
    _, V, F, _ = _single_piece()
    K = Q.lbs_matrix(V, F, np.zeros(F.shape[0], dtype=complex))
    L = cotan_laplacian(V, F)
    assert abs(K - L).max() < 1e-13 * abs(L).max()


def test_solver_reproduces_a_map_from_its_own_coefficients():
    _, V, F, loop = _single_piece()
    z = V[:, 0] + 1j * V[:, 1]
    f = z + 0.2 * np.conj(z) ** 2 + 0.1j * z * np.conj(z)
    mu = Q.beltrami(V, F, f)
    assert not Q.folded(V, F, f).any() and np.abs(mu).max() > 0.1
    g = Q.lbs_solve(V, F, loop, mu, f[loop])
    assert np.abs(g - f).max() < 1e-10


def test_fold_from_a_dragged_vertex_is_removed():
    m, V, F, loop = _single_piece()
    w = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk").final[0]
    assert not Q.folded(V, F, w).any()
    wf = _dragged(V, F, loop, w)
    out, before, rounds, after = Q.fix_piece(V, F, loop, wf)
    assert before > 0 and after == 0 and 1 <= rounds <= 4
    assert np.abs(Q.beltrami(V, F, out)).max() < 1.0
    assert (Q.signed_area(F, out) > 0).all()
    assert np.array_equal(out[loop], wf[loop])
    # the fix lands near the map before the vertex was dragged
    assert np.abs(out - w).max() < 5e-3


def test_fold_next_to_a_concave_boundary_is_removed():
    m = meshgen.polar_disk_mesh(rings=12, sectors=24, jitter=0.0)
    V = m.V.copy()
    V[:, 2] = 0.0
    P = partition(V, m.F, face_labels=np.zeros(m.F.shape[0], dtype=np.int32))
    loop = P.loops[0]
    th = np.angle(V[loop, 0] + 1j * V[loop, 1])
    wb = (1.0 + 0.6 * np.cos(5 * th)) * np.exp(1j * th)
    w = harmonic_solve(cotan_laplacian(V, m.F), loop, wb)
    assert Q.folded(V, m.F, w).sum() > 10     # the harmonic extension folds
    out, before, rounds, after = Q.fix_piece(V, m.F, loop, w)
    assert after == 0 and rounds <= Q.ROUNDS
    assert np.abs(Q.beltrami(V, m.F, out)).max() < 1.0
    assert np.array_equal(out[loop], wb)


def test_fold_free_map_is_unchanged_and_only_folding_pieces_move():
    m = meshgen.heightfield_disk_mesh(3000, seed=3, nx=2, ny=1)
    res = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk")
    P = res.part
    U = res.out.copy()
    fixed, counts = Q.fix_folds(m.V, m.F, P, U)
    assert np.array_equal(fixed, U) and all(c == (0, 0, 0) for c in counts)
    # drag an interior vertex of piece 1 only (not shared with piece 0)
    g1 = P.verts[1]
    loop1 = np.searchsorted(g1, P.loops[1])
    w1 = U[g1, 0] + 1j * U[g1, 1]
    wf = _dragged(m.V[g1], P.local_F[1], loop1, w1)
    moved = g1[np.nonzero(wf != w1)[0]]
    assert moved.size == 1 and moved[0] not in set(P.verts[0].tolist())
    U2 = U.copy()
    U2[moved[0]] = [wf[wf != w1].real[0], wf[wf != w1].imag[0]]
    fixed2, counts2 = Q.fix_folds(m.V, m.F, P, U2)
    assert counts2[0] == (0, 0, 0) and counts2[1][0] > 0 and counts2[1][2] == 0
    assert np.array_equal(fixed2[P.verts[0]], U2[P.verts[0]])
    only1 = np.setdiff1d(g1, P.verts[0])
    assert np.abs(fixed2[only1] - U[only1]).max() < 5e-3
