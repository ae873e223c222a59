"""Area distortion and the Mobius area step (Section 6.2).  Test infrastructure.

Area distortion of a face T under a map phi (Section 6.2 definition):
    d_area(T) = ln( (Area(phi(T)) / sum_T' Area(phi(T'))) / (Area(T) / sum_T' Area(T')) )
with Area(T) the surface triangle's area and Area(phi(T)) the parameter
triangle's area (planar maps; the signed area, which must stay positive).

The area step composes the map with the Mobius transformation f that
minimises mean |d_area| of f o phi, over the families Section 6.2 names:
* disk: the automorphisms f(z) = (z - alpha) / (1 - conj(alpha) z), |alpha| < 1;
* free boundary: the Mobius maps (a z + b) / (c z + d).  Normalised area
  ratios do not change under similarities a z + b, so only the coset of f
  modulo them matters; every coset holds exactly one f_q(z) = z / (1 - q z)
  (q = 0: the identity coset; otherwise the pole 1/q), and f_q o f_p = f_{p+q}.
  The step searches q.  (Reading: the paper optimises all eight real
  parameters; the other six only move the result by a similarity.)
* sphere: tau^-1 o f o tau for a Mobius map f, i.e. a conformal map of the
  sphere; rotations leave chordal areas unchanged, and every such map is a
  rotation after exactly one ball automorphism (Ahlfors' form)
      T_a(x) = ((1 - |a|^2)(x - a) - |x - a|^2 a) / (1 - 2<a, x> + |a|^2 |x|^2),  |a| < 1,
  which keeps the unit sphere (T_0 = id, T_a(a) = 0, T_a(0) = -a).  The step
  searches a in R^3.  Parameter areas on the sphere are those of the chordal
  triangles (the reading of the angle metric), which must face outwards.
The search is Nelder and Mead's simplex method (Computer Journal 7, 1965) on
the real parameters, from the identity, with reflection 1, expansion 2,
contraction 1/2 and shrink 1/2; a parameter that leaves the family's domain
(|alpha| >= 1, |a| >= 1) or gives any face a non-positive area (the pole of f
inside the image) scores +inf.
"""
from __future__ import annotations

import numpy as np

NM_STEP = 0.05       # initial simplex edge
NM_FTOL = 1e-12      # stop when the simplex's objective spread is below this
NM_XTOL = 1e-9       # ... and its size below this
NM_MAXIT = 500


def surface_areas(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    cr = np.cross(b - a, c - a)
    return 0.5 * np.sqrt((cr * cr).sum(axis=1))


def planar_signed_areas(U: np.ndarray, F: np.ndarray) -> np.ndarray:
    a, b, c = U[F[:, 0]], U[F[:, 1]], U[F[:, 2]]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))


def area_distortion(V: np.ndarray, F: np.ndarray, U: np.ndarray) -> np.ndarray:
    """d_area per face of the planar map U (Section 6.2)."""
    at = surface_areas(V, F)
    af = planar_signed_areas(U, F)
    return np.log((af / af.sum()) / (at / at.sum()))


def mobius(variant: str, p: complex, z: np.ndarray) -> np.ndarray:
    """The family member with parameter p applied to complex points z."""
    if variant == "disk":
        return (z - p) / (1.0 - np.conj(p) * z)
    if variant == "free":
        return z / (1.0 - p * z)
    raise ValueError(variant)


def ball_automorphism(a: np.ndarray, X: np.ndarray) -> np.ndarray:
    """T_a on the rows of X (points of R^3)."""
    a = np.asarray(a, dtype=np.float64)
    aa = float(a @ a)
    xa = X @ a
    xx = (X * X).sum(axis=1)
    d = X - a
    dd = (d * d).sum(axis=1)
    num = (1.0 - aa) * d - dd[:, None] * a
    return num / (1.0 - 2.0 * xa + aa * xx)[:, None]


def chordal_areas(X: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Area of each chordal triangle, negative when it faces inwards."""
    a, b, c = X[F[:, 0]], X[F[:, 1]], X[F[:, 2]]
    cr = np.cross(b - a, c - a)
    ar = 0.5 * np.sqrt((cr * cr).sum(axis=1))
    return np.where((cr * (a + b + c)).sum(axis=1) > 0.0, ar, -ar)


def sphere_area_distortion(V: np.ndarray, F: np.ndarray, X: np.ndarray) -> np.ndarray:
    """d_area per face of a spherical map X (chordal parameter triangles)."""
    at = surface_areas(V, F)
    af = chordal_areas(X, F)
    return np.log((af / af.sum()) / (at / at.sum()))


def sphere_objective(V, F, X, a) -> float:
    """mean |d_area| of T_a o X; +inf for |a| >= 1 or an inward-facing triangle."""
    a = np.asarray(a, dtype=np.float64)
    if float(a @ a) >= 1.0:
        return np.inf
    af = chordal_areas(ball_automorphism(a, X), F)
    if not np.all(np.isfinite(af)) or np.any(af <= 0.0):
        return np.inf
    at = surface_areas(V, F)
    d = np.log((af / af.sum()) / (at / at.sum()))
    return float(np.abs(d).mean())


def objective(V, F, U, variant: str, p: complex) -> float:
    """mean |d_area| of f_p o U; +inf outside the family's domain or on a fold."""
    if variant == "disk" and abs(p) >= 1.0:
        return np.inf
    z = mobius(variant, p, U[:, 0] + 1j * U[:, 1])
    W = np.stack([z.real, z.imag], axis=1)
    af = planar_signed_areas(W, F)
    if not np.all(np.isfinite(af)) or np.any(af <= 0.0):
        return np.inf
    at = surface_areas(V, F)
    d = np.log((af / af.sum()) / (at / at.sum()))
    return float(np.abs(d).mean())


def nelder_mead(fun, x0, step=NM_STEP, ftol=NM_FTOL, xtol=NM_XTOL, maxit=NM_MAXIT):
    """Nelder-Mead on R^n: returns (best point, best value, evaluations)."""
    x0 = np.array(x0, dtype=np.float64)
    n = x0.size
    pts = [x0.copy()]
    for i in range(n):
        e = x0.copy()
        e[i] += step
        pts.append(e)
    val = [fun(x) for x in pts]
    evals = n + 1
    w = n                                               # index of the worst after sorting
    for _ in range(maxit):
        order = sorted(range(n + 1), key=lambda i: val[i])
        pts = [pts[i] for i in order]
        val = [val[i] for i in order]
        size = max(np.abs(pts[i] - pts[0]).max() for i in range(1, n + 1))
        if np.isfinite(val[w]) and val[w] - val[0] <= ftol and size <= xtol:
            break
        c = pts[0].copy()                               # centroid of the n best
        for i in range(1, n):
            c = c + pts[i]
        c = c / n
        xr = c + (c - pts[w])                           # reflection
        fr = fun(xr)
        evals += 1
        if fr < val[0]:
            xe = c + 2.0 * (c - pts[w])                 # expansion
            fe = fun(xe)
            evals += 1
            if fe < fr:
                pts[w], val[w] = xe, fe
            else:
                pts[w], val[w] = xr, fr
        elif fr < val[w - 1]:
            pts[w], val[w] = xr, fr
        else:
            if fr < val[w]:                             # outside contraction
                xc = c + 0.5 * (xr - c)
            else:                                       # inside contraction
                xc = c + 0.5 * (pts[w] - c)
            fc = fun(xc)
            evals += 1
            if fc < min(fr, val[w]):
                pts[w], val[w] = xc, fc
            else:                                       # shrink towards the best
                for i in range(1, n + 1):
                    pts[i] = pts[0] + 0.5 * (pts[i] - pts[0])
                    val[i] = fun(pts[i])
                    evals += 1
    i = int(np.argmin(val))
    return pts[i], val[i], evals


def area_step(V, F, U, variant: str):
    """The Mobius area step: (parameter, mean |d_area| before, after, evaluations, mapped U).
    For "sphere" U is [n, 3] on the unit sphere and the parameter is a in R^3."""
    if variant == "sphere":
        before = sphere_objective(V, F, U, np.zeros(3))
        a, after, evals = nelder_mead(lambda x: sphere_objective(V, F, U, x), [0.0, 0.0, 0.0])
        return a, before, after, evals, ball_automorphism(a, U)
    before = objective(V, F, U, variant, 0j)
    x, after, evals = nelder_mead(lambda x: objective(V, F, U, variant, complex(x[0], x[1])), [0.0, 0.0])
    p = complex(x[0], x[1])
    z = mobius(variant, p, U[:, 0] + 1j * U[:, 1])
    return p, before, after, evals, np.stack([z.real, z.imag], axis=1)
