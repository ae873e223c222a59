"""Fold-over fix by quasi-conformal composition (Section 4.5 and Algorithm 3's
last step; Beltrami coefficient and composition formula, Section 3.5).
Test infrastructure.

A piecewise linear map phi of a piece is folding-free iff |mu_phi| < 1 on
every face (Section 3.5: J = |phi_z|^2 (1 - |mu|^2)).  Algorithm 3 checks
mu of the final map of every piece and, where it folds, composes the map with
a quasi-conformal map chosen through the composition formula so that the
composition has a Beltrami coefficient of modulus below 1 and is therefore
folding-free.

Readings (the same in the CUDA library):
* mu of a face is that of the affine map from the surface triangle, laid flat
  in its own orthonormal frame (p0 at 0, p1 on +x), to the parameter triangle:
  mu = f_zbar / f_z.  The inverse map has the same |mu|, so the check of
  Algorithm 3 on mu of the inverse is the check |mu| >= 1 - 1e-6 (or a signed
  area <= 0) here.
* A map with Beltrami coefficient nu and the piece's welded boundary values is
  the solution of the linear Beltrami solver: div(A_nu grad u) = 0 and
  div(A_nu grad v) = 0 for phi = u + i v, with
      A_nu = [[(rho-1)^2 + tau^2, -2 tau], [-2 tau, (rho+1)^2 + tau^2]] / (1 - |nu|^2),
  nu = rho + i tau, discretised with linear elements on the surface
  triangles (each in its own flat frame).  With nu = 0 the element matrices
  are the cotangent stiffness matrices; with nu = mu_phi on every face the
  solution is phi itself (exact for piecewise linear maps), so a composition
  changes the map only where nu differs from mu_phi.
* The composition of Algorithm 3 (the paper gives no discrete recipe) runs in
  rounds t = 1 .. ROUNDS on a piece that folds.  The fold region is the folded
  faces grown by t rings of faces that share a vertex; the composition's
  coefficient nu is mu_phi outside the region and mu_phi with its modulus
  capped at KAPPA inside it (the composition formula with phi_2 removing the
  excess distortion, Section 3.5); the new map is the solver's solution for nu
  with the boundary kept.  The rounds stop as soon as no face folds.
  KAPPA = 0.7: a cap near 1 leaves dragged vertices in place, a cap near 0
  forbids the dilatation a fold next to a concave boundary needs; 0.7 fixes
  both kinds in the pinned cases.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.linalg import spsolve

FOLD_THRESH = 1e-6   # a face folds when |mu| >= 1 - FOLD_THRESH (or its signed area <= 0)
KAPPA = 0.7          # cap of |nu| inside the fold region
ROUNDS = 16          # compositions at most


def face_frames(V: np.ndarray, F: np.ndarray):
    """Each surface triangle in its own orthonormal frame: (l1, x2, y2) with
    p0 -> (0, 0), p1 -> (l1, 0), p2 -> (x2, y2), y2 > 0."""
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1 = p1 - p0
    e2 = p2 - p0
    l1 = np.linalg.norm(e1, axis=1)
    x2 = (e1 * e2).sum(axis=1) / l1
    y2 = np.linalg.norm(np.cross(e1, e2), axis=1) / l1
    return l1, x2, y2


def beltrami(V: np.ndarray, F: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Complex mu = f_zbar / f_z of the affine map of every face (w: complex
    image of every vertex)."""
    l1, x2, y2 = face_frames(V, F)
    w0 = w[F[:, 0]]
    w1 = w[F[:, 1]] - w0
    w2 = w[F[:, 2]] - w0
    fx = w1 / l1
    fy = (w2 - w1 * x2 / l1) / y2
    fz = 0.5 * (fx - 1j * fy)
    fzb = 0.5 * (fx + 1j * fy)
    return fzb / fz


def signed_area(F: np.ndarray, w: np.ndarray) -> np.ndarray:
    a, b, c = w[F[:, 0]], w[F[:, 1]], w[F[:, 2]]
    return 0.5 * ((b - a).real * (c - a).imag - (b - a).imag * (c - a).real)


def folded(V: np.ndarray, F: np.ndarray, w: np.ndarray) -> np.ndarray:
    return (signed_area(F, w) <= 0.0) | (np.abs(beltrami(V, F, w)) >= 1.0 - FOLD_THRESH)


def fold_region(F: np.ndarray, n: int, bad: np.ndarray, rings: int) -> np.ndarray:
    """The faces within `rings` rings (faces sharing a vertex) of the bad faces."""
    reg = bad.copy()
    for _ in range(rings):
        mark = np.zeros(n, dtype=bool)
        mark[F[reg].ravel()] = True
        reg = mark[F].any(axis=1)
    return reg


def target_coefficient(mu: np.ndarray, region: np.ndarray) -> np.ndarray:
    """nu: mu outside the region; inside, mu with its modulus capped at KAPPA."""
    nu = mu.copy()
    a = np.abs(mu)
    cap = region & (a > KAPPA)
    nu[cap] = KAPPA * mu[cap] / a[cap]
    return nu


def lbs_matrix(V: np.ndarray, F: np.ndarray, nu: np.ndarray):
    """Linear-element matrix of div(A_nu grad .) on the surface triangles:
    K_jk = sum over faces of area * grad(phi_j)^T A_nu grad(phi_k), gradients
    in each face's flat frame.  Positive semidefinite; rows sum to 0."""
    n = V.shape[0]
    l1, x2, y2 = face_frames(V, F)
    area = 0.5 * l1 * y2
    P = np.stack([np.zeros_like(l1), np.zeros_like(l1), l1, np.zeros_like(l1), x2, y2], axis=1).reshape(-1, 3, 2)
    # gradient of the hat function of corner c: rotate the opposite edge, / (2 area)
    G = np.empty((F.shape[0], 3, 2))
    for c in range(3):
        e = P[:, (c + 2) % 3] - P[:, (c + 1) % 3]
        G[:, c, 0] = -e[:, 1] / (2.0 * area)
        G[:, c, 1] = e[:, 0] / (2.0 * area)
    rho, tau = nu.real, nu.imag
    den = 1.0 - np.abs(nu) ** 2
    a1 = ((rho - 1.0) ** 2 + tau ** 2) / den
    a2 = -2.0 * tau / den
    a3 = ((rho + 1.0) ** 2 + tau ** 2) / den
    rows, cols, vals = [], [], []
    for j in range(3):
        AGj0 = a1 * G[:, j, 0] + a2 * G[:, j, 1]
        AGj1 = a2 * G[:, j, 0] + a3 * G[:, j, 1]
        for k in range(3):
            rows.append(F[:, j])
            cols.append(F[:, k])
            vals.append(area * (AGj0 * G[:, k, 0] + AGj1 * G[:, k, 1]))
    K = coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    K.sum_duplicates()
    return K


def lbs_solve(V: np.ndarray, F: np.ndarray, loop: np.ndarray, nu: np.ndarray, wb: np.ndarray) -> np.ndarray:
    """The map with Beltrami coefficient nu and boundary values wb on loop."""
    n = V.shape[0]
    K = lbs_matrix(V, F, nu)
    isb = np.zeros(n, dtype=bool)
    isb[loop] = True
    I = np.nonzero(~isb)[0]
    w = np.zeros(n, dtype=np.complex128)
    w[loop] = wb
    if I.size:
        KII = K[I][:, I].tocsc()
        KIB = K[I][:, loop]
        w[I] = spsolve(KII, -(KIB @ wb.real)) + 1j * spsolve(KII, -(KIB @ wb.imag))
    return w


def fix_piece(V: np.ndarray, F: np.ndarray, loop: np.ndarray, w: np.ndarray):
    """Algorithm 3's fold check and fix on one piece (local ids).  Returns the
    new map, the number of faces that folded before, the compositions made and
    the faces that still fold after them."""
    cur = w.copy()
    bad = folded(V, F, cur)
    before = int(bad.sum())
    t = 0
    while bad.any() and t < ROUNDS:
        t += 1
        nu = target_coefficient(beltrami(V, F, cur), fold_region(F, V.shape[0], bad, t))
        cur = lbs_solve(V, F, loop, nu, cur[loop])
        bad = folded(V, F, cur)
    return cur, before, t, int(bad.sum())


def fix_folds(V: np.ndarray, F: np.ndarray, part, U: np.ndarray):
    """The fix on every piece of a planar result U [nv, 2] (free or disk
    variant), boundary values kept; the gather takes the lowest-label piece's
    copy.  Returns (new U, per piece (folded before, compositions, folded
    after))."""
    out = np.full(U.shape, np.nan)
    counts = []
    w_all = U[:, 0] + 1j * U[:, 1]
    for i in range(part.K):
        g = part.verts[i]
        loop = np.searchsorted(g, part.loops[i])
        w, nb, t, na = fix_piece(V[g], part.local_F[i], loop, w_all[g])
        counts.append((nb, t, na))
        have = ~np.isnan(out[g, 0])
        out[g[~have], 0] = w.real[~have]
        out[g[~have], 1] = w.imag[~have]
    return out, counts
