"""Pins for the oracle's cotangent Laplacian and DNCP (Section 4.2).

Checked against: an independent dense P1 finite-element stiffness assembly,
linear precision on planar meshes, u^T L u = 2 Area, E_C(identity) = 0 on a
planar mesh (which fixes the area-matrix constant), E_C >= 0, similarity
reproduction, and dense brute-force solves on small meshes.
"""
import numpy as np
import pytest

from oracle.laplacian import cotan_laplacian
from oracle.dncp import dncp, dncp_matrix, area_matrix, boundary_area, pins
from oracle.mesh import partition
from oracle.pipeline import harmonic_solve
from paper_1903_12359_gb300 import meshgen


def _piece(m, i=0, planar=False):
    P = partition(m.V, m.F, face_labels=m.face_labels)
    X = m.V[P.verts[i]].copy()
    if planar:
        X[:, 2] = 0.0
    ll = np.searchsorted(P.verts[i], P.loops[i])
    return X, P.local_F[i], ll


def _fem_stiffness(X, Fl):
    """Dense P1 stiffness: sum over triangles of area * grad(phi_a) . grad(phi_b)."""
    n = X.shape[0]
    K = np.zeros((n, n))
    for t in Fl:
        p = X[t]
        e1, e2 = p[1] - p[0], p[2] - p[0]
        nrm = np.cross(e1, e2)
        area = 0.5 * np.linalg.norm(nrm)
        u = e1 / np.linalg.norm(e1)
        v = np.cross(nrm / np.linalg.norm(nrm), u)
        q = np.array([[0.0, 0.0], [e1 @ u, e1 @ v], [e2 @ u, e2 @ v]])
        A = np.column_stack([np.ones(3), q])
        G = np.linalg.inv(A)[1:, :]            # rows: d/dx, d/dy of the 3 hat functions
        K[np.ix_(t, t)] += area * (G.T @ G)
    return K


def test_cotan_matches_fem_and_is_psd():
    m = meshgen.polar_disk_mesh(rings=6, sectors=12, seed=3)
    X, Fl, _ = _piece(m)
    L = cotan_laplacian(X, Fl).toarray()
    K = _fem_stiffness(X, Fl)
    assert np.abs(L - K).max() < 1e-12 * np.abs(K).max()
    assert np.abs(L - L.T).max() == 0.0
    assert np.abs(L.sum(axis=1)).max() < 1e-13 * np.abs(L).max()
    assert np.linalg.eigvalsh(L).min() > -1e-12


def test_linear_precision_and_area():
    m = meshgen.heightfield_disk_mesh(1500, seed=0, nx=2, ny=1)
    X, Fl, ll = _piece(m, planar=True)
    L = cotan_laplacian(X, Fl)
    n = X.shape[0]
    interior = np.setdiff1d(np.arange(n), ll)
    for c in (0, 1):
        assert np.abs((L @ X[:, c])[interior]).max() < 1e-12
    area = 0.5 * np.abs(np.cross(X[Fl[:, 1]] - X[Fl[:, 0]], X[Fl[:, 2]] - X[Fl[:, 0]])[:, 2]).sum()
    e = X[:, 0] @ (L @ X[:, 0]) + X[:, 1] @ (L @ X[:, 1])
    assert abs(e - 2 * area) < 1e-12 * area
    # Dirichlet problem with identity boundary returns the identity
    z = X[:, 0] + 1j * X[:, 1]
    u = harmonic_solve(L, ll, z[ll])
    assert np.abs(u - z).max() < 1e-12


def test_area_constant_gives_zero_conformal_energy_on_planar_identity():
    m = meshgen.heightfield_disk_mesh(1500, seed=1, nx=2, ny=1)
    X, Fl, ll = _piece(m, planar=True)
    L = cotan_laplacian(X, Fl)
    U = np.concatenate([X[:, 0], X[:, 1]])
    A = boundary_area(X[:, 0] + 1j * X[:, 1], ll)
    Q = dncp_matrix(L, ll)
    assert abs(0.5 * U @ (Q @ U)) < 1e-12 * A            # E_C(identity) = 0
    assert abs(U @ (area_matrix(X.shape[0], ll) @ U) - 2 * A) < 1e-12 * A
    assert np.abs(Q @ U).max() < 1e-11                    # identity is stationary
    # the paper's printed constant (+-1) would leave E_C = -A, not 0
    E1 = 0.5 * (U @ (np.concatenate([L @ X[:, 0], L @ X[:, 1]]))) - 0.5 * (U @ (2 * area_matrix(X.shape[0], ll) @ U))
    assert abs(E1 + A) < 1e-10 * A


def test_dncp_reproduces_planar_similarity():
    m = meshgen.heightfield_disk_mesh(1500, seed=2, nx=2, ny=1)
    X, Fl, ll = _piece(m, planar=True)
    u, ref = dncp(X, Fl, ll)
    z = X[:, 0] + 1j * X[:, 1]
    M = np.column_stack([z, np.ones_like(z)])
    coef, *_ = np.linalg.lstsq(M, u, rcond=None)
    assert np.abs(M @ coef - u).max() < 1e-10
    assert ref >= 0 and abs(u[ref]) == 0.0
    p0, p1 = pins(ll)
    assert abs((u[p1] - u[p0]) - 1.0) < 1e-12


def test_dncp_energy_psd_and_dense_bruteforce():
    m = meshgen.polar_disk_mesh(rings=5, sectors=16, seed=1)   # 81 vertices
    X, Fl, ll = _piece(m)
    L = cotan_laplacian(X, Fl)
    Q = dncp_matrix(L, ll).toarray()
    ev = np.linalg.eigvalsh(Q)
    assert ev.min() > -1e-12 * ev.max()
    assert (ev < 1e-10 * ev.max()).sum() == 2            # translations (curved piece)
    Xp = X.copy()
    Xp[:, 2] = 0.0
    evp = np.linalg.eigvalsh(dncp_matrix(cotan_laplacian(Xp, Fl), ll).toarray())
    assert (evp < 1e-10 * evp.max()).sum() == 4          # planar: all similarities are conformal
    n = X.shape[0]
    u, ref = dncp(X, Fl, ll, L)
    p0, p1 = pins(ll)
    fixed = [p0, p1, n + p0, n + p1]
    free = np.setdiff1d(np.arange(2 * n), fixed)
    ufix = np.array([0.0, 1.0, 0.0, 0.0])
    sol = np.linalg.solve(Q[np.ix_(free, free)], -Q[np.ix_(free, fixed)] @ ufix)
    U = np.zeros(2 * n)
    U[fixed] = ufix
    U[free] = sol
    ud = U[:n] + 1j * U[n:]
    ud = ud - ud[ref]
    assert np.abs(ud - u).max() < 1e-12
