"""Cotangent Laplacian (Section 4.2, the L^cotan definition) -- test infrastructure.

For every edge (p, q) with opposite angles alpha, beta inside the piece the
weight is w_pq = (cot alpha + cot beta) / 2 (one term on a boundary edge).

Reading: the paper prints off-diagonal +w and diagonal -sum, a negative
semidefinite matrix, while calling it positive definite; only the sign differs
and the Laplace solutions are the same.  We store the positive semidefinite
form L_pq = -w_pq, L_pp = sum_q w_pq, so u^T L u = sum_edges w |u_p - u_q|^2,
which for a P1 finite element map is the integral of |grad u|^2.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix, csr_matrix

from .common import OracleError


def corner_cotangents(X: np.ndarray, Fl: np.ndarray) -> np.ndarray:
    """cot of the angle at each corner: cot = (e1 . e2) / |e1 x e2| (FP64).

    Returns [nf, 3]: column c is the corner at vertex Fl[:, c].
    """
    out = np.empty((Fl.shape[0], 3))
    for c in range(3):
        p = X[Fl[:, c]]
        q = X[Fl[:, (c + 1) % 3]]
        r = X[Fl[:, (c + 2) % 3]]
        e1 = q - p
        e2 = r - p
        dot = (e1 * e2).sum(axis=1)
        cr = np.cross(e1, e2)
        nrm = np.sqrt((cr * cr).sum(axis=1))
        if np.any(nrm == 0.0):
            raise OracleError("DEGENERATE", "zero-area face")
        out[:, c] = dot / nrm
    return out


def cotan_laplacian(X: np.ndarray, Fl: np.ndarray) -> csr_matrix:
    """PSD cotangent Laplacian of one piece (local vertex ids)."""
    n = X.shape[0]
    cot = corner_cotangents(X, Fl)
    rows, cols, vals = [], [], []
    for c in range(3):
        # the corner at vertex c is opposite the edge (c+1, c+2)
        i = Fl[:, (c + 1) % 3]
        j = Fl[:, (c + 2) % 3]
        w = 0.5 * cot[:, c]
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [-w, -w, w, w]
    L = coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    L.sum_duplicates()
    L.sort_indices()
    return L


def csr_pattern(L: csr_matrix):
    """Row pointers and column indices (sorted, diagonal stored)."""
    return L.indptr.astype(np.int64), L.indices.astype(np.int64)
