"""Angle distortion and fold checks (Section 5; Section 3.5; Section 4.5).

Test infrastructure.  The angular distortion of the corner [v_i, v_j, v_k] is
d = angle(phi(v_i), phi(v_j), phi(v_k)) - angle(v_i, v_j, v_k) in degrees,
each angle computed as atan2(|e1 x e2|, e1 . e2).  Statistics over |d|: mean,
population standard deviation, median and inter-quartile range (linear
interpolation, numpy's default), and maximum.  For a spherical result the
parameter-domain angle is that of the chordal triangle on the unit sphere.

Folds (Section 3.5): a map is folding-free iff |mu| < 1; for a piecewise
linear map a face folds iff its signed area is <= 0.  The check flags faces
with signed area <= 0 or |mu| >= 1 - 1e-6.
"""
from __future__ import annotations

import numpy as np


def corner_angles(X: np.ndarray, F: np.ndarray) -> np.ndarray:
    """[nf, 3] angle at corner c (vertex F[:, c]) in radians; X is [n, 2] or [n, 3]."""
    out = np.empty(F.shape)
    X3 = X if X.shape[1] == 3 else np.concatenate([X, np.zeros((X.shape[0], 1))], axis=1)
    for c in range(3):
        p = X3[F[:, c]]
        e1 = X3[F[:, (c + 1) % 3]] - p
        e2 = X3[F[:, (c + 2) % 3]] - p
        cr = np.cross(e1, e2)
        out[:, c] = np.arctan2(np.sqrt((cr * cr).sum(axis=1)), (e1 * e2).sum(axis=1))
    return out


def angle_distortion(V: np.ndarray, F: np.ndarray, U: np.ndarray) -> dict:
    d = np.degrees(corner_angles(U, F) - corner_angles(V, F)).ravel()
    a = np.abs(d)
    q1, med, q3 = np.percentile(a, [25.0, 50.0, 75.0])
    return {"mean": float(a.mean()), "sd": float(a.std()), "median": float(med),
            "iqr": float(q3 - q1), "max": float(a.max()), "n": int(a.size)}


def signed_areas(U: np.ndarray, F: np.ndarray) -> np.ndarray:
    a, b, c = U[F[:, 0]], U[F[:, 1]], U[F[:, 2]]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))


def beltrami_abs(V: np.ndarray, F: np.ndarray, U: np.ndarray) -> np.ndarray:
    """|mu| of the piecewise linear map from each surface triangle to the plane.

    The triangle is laid flat in its own orthonormal frame (p0 at 0, p1 on the
    +x axis); the affine map's complex derivatives give mu = f_zbar / f_z.
    |mu| of the inverse map equals |mu| of the map.
    """
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1 = p1 - p0
    e2 = p2 - p0
    l1 = np.linalg.norm(e1, axis=1)
    x2 = (e1 * e2).sum(axis=1) / l1
    cr = np.cross(e1, e2)
    y2 = np.linalg.norm(cr, axis=1) / l1
    w0 = U[F[:, 0], 0] + 1j * U[F[:, 0], 1]
    w1 = U[F[:, 1], 0] + 1j * U[F[:, 1], 1] - w0
    w2 = U[F[:, 2], 0] + 1j * U[F[:, 2], 1] - w0
    # f(x, y) = w1 * (x - x2 y / y2)/l1 + w2 * y / y2 in the flat frame
    fx = w1 / l1
    fy = (w2 - w1 * x2 / l1) / y2
    fz = 0.5 * (fx - 1j * fy)
    fzb = 0.5 * (fx + 1j * fy)
    return np.abs(fzb) / np.abs(fz)


def fold_check(V: np.ndarray, F: np.ndarray, U: np.ndarray, thresh: float = 1e-6) -> dict:
    sa = signed_areas(U, F)
    mu = beltrami_abs(V, F, U)
    bad = (sa <= 0.0) | (mu >= 1.0 - thresh)
    return {"flips": int((sa <= 0.0).sum()), "folds": int(bad.sum()), "max_mu": float(mu.max())}
