"""Local conformal parameterization by DNCP (Section 4.2) -- test infrastructure.

DNCP minimises E_C(u) = E_D(u) - A(u) with two boundary vertices pinned, which
is the linear system ((L (+) L) - M^area) [x; y] = 0 on the free unknowns.

Readings (the same in the CUDA library):
* With L positive semidefinite (see ``laplacian``), E_D = 1/2 [x;y]^T (L(+)L) [x;y].
  The area term must satisfy [x;y]^T M [x;y] = 2 A(u) so that E_C vanishes on a
  planar identity map; the paper's entries +-1 give 4 A, so M carries +-1/2.
  For a boundary edge p -> q (loop order): M[p, n+q] = M[n+q, p] = +1/2 and
  M[q, n+p] = M[n+p, q] = -1/2.
* Pins: loop position 0 at (0, 0) and loop position floor(b/2) at (1, 0).
* Local frame: afterwards the piece is translated so that its reference vertex
  -- the first interior vertex at or after local index floor(n/2), wrapping --
  sits at 0.  That makes the auxiliary point "0" of Algorithm 2 an interior
  point of the piece's image.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix, bmat
from scipy.sparse.linalg import spsolve

from .laplacian import cotan_laplacian


def area_matrix(n: int, loop_local: np.ndarray):
    """M^area as a 2n x 2n sparse matrix with entries +-1/2."""
    p = loop_local
    q = np.roll(loop_local, -1)
    rows = np.concatenate([p, n + q, q, n + p])
    cols = np.concatenate([n + q, p, n + p, q])
    vals = np.concatenate([np.full(p.size, 0.5), np.full(p.size, 0.5),
                           np.full(p.size, -0.5), np.full(p.size, -0.5)])
    return coo_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n)).tocsr()


def dncp_matrix(L, loop_local: np.ndarray):
    n = L.shape[0]
    return (bmat([[L, None], [None, L]]) - area_matrix(n, loop_local)).tocsr()


def boundary_area(u: np.ndarray, loop_local: np.ndarray) -> float:
    """A(u) = 1/2 sum over boundary edges p -> q of (x_p y_q - y_p x_q)."""
    p = loop_local
    q = np.roll(loop_local, -1)
    return 0.5 * float(np.sum(u[p].real * u[q].imag - u[p].imag * u[q].real))


def pins(loop_local: np.ndarray):
    return int(loop_local[0]), int(loop_local[loop_local.size // 2])


def reference_vertex(n: int, loop_local: np.ndarray) -> int:
    """First interior local vertex at or after floor(n/2), wrapping around."""
    on_loop = np.zeros(n, dtype=bool)
    on_loop[loop_local] = True
    for t in range(n):
        v = (n // 2 + t) % n
        if not on_loop[v]:
            return v
    return -1   # a piece without interior vertices


def dncp(X: np.ndarray, Fl: np.ndarray, loop_local: np.ndarray, L=None):
    """Solve DNCP for one piece; returns complex local coordinates (all vertices).

    The result is translated so the reference vertex is at 0 (when the piece has
    an interior vertex).
    """
    if L is None:
        L = cotan_laplacian(X, Fl)
    n = L.shape[0]
    Q = dncp_matrix(L, loop_local)
    p0, p1 = pins(loop_local)
    fixed = np.array([p0, p1, n + p0, n + p1])
    ufix = np.array([0.0, 1.0, 0.0, 0.0])
    free = np.ones(2 * n, dtype=bool)
    free[fixed] = False
    fi = np.nonzero(free)[0]
    Qff = Q[fi][:, fi].tocsc()
    rhs = -(Q[fi][:, fixed] @ ufix)
    sol = spsolve(Qff, rhs)
    U = np.zeros(2 * n)
    U[fixed] = ufix
    U[fi] = sol
    u = U[:n] + 1j * U[n:]
    ref = reference_vertex(n, loop_local)
    if ref >= 0:
        u = (u.real - u[ref].real) + 1j * (u.imag - u[ref].imag)
    return u, ref
