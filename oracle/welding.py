"""Zipper maps, intermediate form and partial welding (Sections 3.4, 4.3, 4.4).

Test infrastructure.  Points are extended complex numbers held as float64
arrays (re, im) plus an infinity flag.  All arithmetic is spelled out on reals
so the order of every rounding is visible (no numpy complex division or abs).

Elementary maps (records):
  SQRT_RATIO  g_1(z) = sqrt((z - z1) / (z - z0))                    (Sec. 3.4)
  OPEN        g_j(z) = sqrt(L_xi(z)^2 - 1),
              L_xi(z) = (Re xi/|xi|^2) z / (1 + (Im xi/|xi|^2) z i) (Sec. 3.4)
  MOB_POLE    g_{k+1}(z) = z / (1 - z/p)                            (Alg. 1)
  CLOSE       h_j(z) = sqrt(T(z)^2 + 1),
              T(z) = z / (-2ab/(a-b) - (a+b)/(a-b) z i)             (Sec. 4.3.2)
  POLE_SQ     h_0(z) = (z / (1 - z/p))^2  (also the geodesic final map)
  MOBIUS      (a z + b) / (c z + d)  (normalisation, disk frame, sphere frame)

Square roots.  Points in the open right half-plane take the principal root
(Kahan-style formula, own |z|).  Points the algorithm has already put on the
imaginary axis (known by their index, never by the sign of a rounding-level
real part) take the root on their own side of the axis: the root whose
imaginary part has the sign of Im of the Mobius image (the map is continuous
from the right half-plane, where the region lies).  The one point that lands
on the branch point itself (the previous zip point, at 0) takes the
sequence's branch, +i or -i (Algorithm 1's "choice of branching").

Conditioning.  The zipper is evaluated in plain FP64 in the paper's order.
On seams that follow straight vertex rows the intermediate form agrees with a
60-digit evaluation to ~1e-11 (relative) at k ~ 400; on zig-zag seams (faces
assigned by centroid on an irregular mesh) boundary points come within 1e-5 of
the imaginary axis and FP64 loses the ordering of the arc (the oracle then
raises NUMERIC).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .common import OracleError

# point modes used while building a chain (phase 1); everything else is PRINCIPAL
PRINCIPAL, SIGN, BRANCH, ZERO, INF = 0, 1, 2, 3, 4

SQRT_RATIO, OPEN, MOB_POLE, CLOSE, POLE_SQ, MOBIUS = range(6)


@dataclass
class Rec:
    kind: int
    p: tuple                 # real parameters of the map
    branch: float = 1.0


class Pts:
    """Extended complex points: float64 (re, im) and a bool infinity flag."""

    def __init__(self, re, im, inf=None):
        self.re = np.array(re, dtype=np.float64).reshape(-1)
        self.im = np.array(im, dtype=np.float64).reshape(-1)
        n = self.re.size
        self.inf = np.zeros(n, dtype=bool) if inf is None else np.array(inf, dtype=bool).reshape(-1)

    @staticmethod
    def from_complex(z, inf=None):
        z = np.asarray(z, dtype=np.complex128).reshape(-1)
        return Pts(z.real.copy(), z.imag.copy(), inf)

    def copy(self):
        return Pts(self.re, self.im, self.inf)

    def take(self, idx):
        return Pts(self.re[idx], self.im[idx], self.inf[idx])

    def complex(self):
        return self.re + 1j * self.im

    def __len__(self):
        return self.re.size


# ---------------------------------------------------------------- arithmetic

def _f(t):
    return np.asarray(t, dtype=np.float64)


def _cdiv(ar, ai, br, bi):
    """(ar + i ai) / (br + i bi) by Smith's algorithm (1962)."""
    ar, ai, br, bi = _f(ar), _f(ai), _f(br), _f(bi)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        big = np.abs(br) >= np.abs(bi)
        r1 = bi / br
        d1 = br + bi * r1
        x1 = (ar + ai * r1) / d1
        y1 = (ai - ar * r1) / d1
        r2 = br / bi
        d2 = br * r2 + bi
        x2 = (ar * r2 + ai) / d2
        y2 = (ai * r2 - ar) / d2
    return np.where(big, x1, x2), np.where(big, y1, y2)


def _cmul(ar, ai, br, bi):
    ar, ai, br, bi = _f(ar), _f(ai), _f(br), _f(bi)
    return ar * br - ai * bi, ar * bi + ai * br


def _hypot(x, y):
    ax = np.abs(x)
    ay = np.abs(y)
    m = np.maximum(ax, ay)
    n = np.minimum(ax, ay)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = n / m
        h = m * np.sqrt(1.0 + q * q)
    return np.where(m == 0.0, 0.0, h)


def _csqrt(x, y):
    """Principal square root (Re >= 0), after Kahan 1987."""
    x, y = _f(x), _f(y)
    h = _hypot(x, y)
    t = np.sqrt((np.abs(x) + h) * 0.5)
    with np.errstate(divide="ignore", invalid="ignore"):
        t2 = t + t
        pr = np.where(x >= 0.0, t, np.abs(y) / t2)
        pi = np.where(x >= 0.0, y / t2, np.copysign(t, y))
    zero = (x == 0.0) & (y == 0.0)
    return np.where(zero, 0.0, pr), np.where(zero, y, pi)


def _root(wr, wi, sr, si, mode, branch):
    """sqrt(w) with the per-point rules; (sr, si) is the pre-square Mobius image."""
    rr, ri = _csqrt(wr, wi)
    flip = (mode == SIGN) & (ri * si < 0.0)
    rr = np.where(flip, -rr, rr)
    ri = np.where(flip, -ri, ri)
    br = mode == BRANCH
    rr = np.where(br, 0.0, rr)
    ri = np.where(br, branch, ri)
    zero = mode == ZERO
    rr = np.where(zero, 0.0, rr)
    ri = np.where(zero, 0.0, ri)
    return rr, ri


# ---------------------------------------------------------------- map records

def rec_sqrt_ratio(z0: complex, z1: complex) -> Rec:
    return Rec(SQRT_RATIO, (z0.real, z0.imag, z1.real, z1.imag))


def _mob_open(cr, ci, zr, zi):
    """Denominator 1 + ci z i and L(z) of the OPEN map."""
    Dr, Di = 1.0 - ci * zi, ci * zr
    Lr, Li = _cdiv(cr * zr, cr * zi, Dr, Di)
    return Dr, Di, Lr, Li


def _mob_close(c1, c2, zr, zi):
    """Denominator c1 - c2 z i and T(z) of the CLOSE map."""
    Dr, Di = c1 + c2 * zi, -(c2 * zr)
    Tr, Ti = _cdiv(zr, zi, Dr, Di)
    return Dr, Di, Tr, Ti


def rec_open(xr: float, xi: float, branch: float) -> Rec:
    s = xr * xr + xi * xi
    return Rec(OPEN, (xr / s, xi / s), branch)


def rec_mob_pole(pr: float, pi: float) -> Rec:
    return Rec(MOB_POLE, (pr, pi))


def rec_close(a: float, b: float) -> Rec:
    """h_j from alpha = a i, beta = b i.

    The paper states the common case a > 0 > b.  Once the shared point has
    wrapped past infinity, beta can lie on the upper axis beyond alpha (or
    alpha on the lower axis); T still takes {alpha, 0, beta} to {i, 0, -i} and
    keeps the right half-plane exactly when c1 = -2ab/(a-b) > 0, which is the
    condition checked here.
    """
    amb = a - b
    c1 = ((-2.0 * a) * b) / amb
    c2 = (a + b) / amb
    if not (amb != 0.0 and c1 > 0.0 and np.isfinite(c1) and np.isfinite(c2) and c2 != 0.0):
        raise OracleError("NUMERIC", f"closing map: alpha={a}i, 0, beta={b}i out of order")
    return Rec(CLOSE, (c1, c2))


def rec_pole_sq(pr: float, pi: float) -> Rec:
    return Rec(POLE_SQ, (pr, pi))


def rec_mobius(a: complex, b: complex, c: complex, d: complex) -> Rec:
    return Rec(MOBIUS, (a.real, a.imag, b.real, b.imag, c.real, c.imag, d.real, d.imag))


def rec_normalize(p1: complex, p2: complex, p3: complex) -> Rec:
    """Mobius taking p1 -> -1, p2 -> 1, p3 -> inf (Algorithm 2, last step):
    T(z) = 2 (z - p1)(p2 - p3) / ((z - p3)(p2 - p1)) - 1."""
    ur, ui = p2.real - p3.real, p2.imag - p3.imag
    vr, vi = p2.real - p1.real, p2.imag - p1.imag
    tr, ti = ur + ur, ui + ui
    ar, ai = tr - vr, ti - vi
    vp3r, vp3i = (float(t) for t in _cmul(vr, vi, p3.real, p3.imag))
    tp1r, tp1i = (float(t) for t in _cmul(tr, ti, p1.real, p1.imag))
    br, bi = vp3r - tp1r, vp3i - tp1i
    return Rec(MOBIUS, (ar, ai, br, bi, vr, vi, -vp3r, -vp3i))


def rec_sphere_frame(p1: complex, p2: complex, q: complex, invert: bool) -> Rec:
    """Mobius taking p1 -> 0, p2 -> inf, q -> 1 (closed weld normalisation);
    ``invert`` gives its reciprocal, the chart w = 1/z used for the piece
    holding infinity."""
    ar, ai = q.real - p2.real, q.imag - p2.imag      # a = q - p2
    cr, ci = q.real - p1.real, q.imag - p1.imag      # c = q - p1
    br, bi = (float(t) for t in _cmul(ar, ai, p1.real, p1.imag))   # b = -p1 (q - p2)
    dr, di = (float(t) for t in _cmul(cr, ci, p2.real, p2.imag))   # d = -p2 (q - p1)
    a, b = complex(ar, ai), complex(-br, -bi)
    c, d = complex(cr, ci), complex(-dr, -di)
    if invert:
        a, b, c, d = c, d, a, b
    return rec_mobius(a, b, c, d)


def rec_half_plane_to_disk(cr: float, ci: float) -> Rec:
    """w -> (w - c) / (w - conj(c)): upper half-plane onto the unit disk, c -> 0,
    infinity -> 1."""
    return rec_mobius(1 + 0j, complex(-cr, -ci), 1 + 0j, complex(-cr, ci))


# ---------------------------------------------------------------- application

def apply_rec(rec: Rec, P: Pts, mode=None) -> Pts:
    """Apply one elementary map to all points; ``mode`` holds per-point rules."""
    n = len(P)
    if mode is None:
        mode = np.zeros(n, dtype=np.int8)
    zr, zi, zinf = P.re, P.im, P.inf
    fin = ~zinf
    outinf = np.zeros(n, dtype=bool)
    k = rec.kind
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        if k == SQRT_RATIO:
            z0r, z0i, z1r, z1i = rec.p
            wr, wi = _cdiv(zr - z1r, zi - z1i, zr - z0r, zi - z0i)
            wr = np.where(fin, wr, 1.0)
            wi = np.where(fin, wi, 0.0)
            outr, outi = _csqrt(wr, wi)
        elif k in (OPEN, CLOSE):
            if k == OPEN:
                cr, ci = rec.p
                _, _, Mr, Mi = _mob_open(cr, ci, zr, zi)
                Minf_i = -(np.float64(cr) / np.float64(ci))   # IEEE: a real xi sends infinity to infinity
            else:
                c1, c2 = rec.p
                _, _, Mr, Mi = _mob_close(c1, c2, zr, zi)
                Minf_i = np.float64(1.0) / np.float64(c2)
            Mr = np.where(fin, Mr, 0.0)
            Mi = np.where(fin, Mi, Minf_i)
            sr = Mr * Mr - Mi * Mi
            si = Mr * Mi + Mi * Mr
            wr = sr - 1.0 if k == OPEN else sr + 1.0
            outr, outi = _root(wr, si, Mr, Mi, mode, rec.branch)
        elif k in (MOB_POLE, POLE_SQ):
            pr, pi = rec.p
            tr, ti = _cdiv(zr, zi, pr, pi)
            Mr, Mi = _cdiv(zr, zi, 1.0 - tr, -ti)
            Mr = np.where(fin, Mr, -pr)
            Mi = np.where(fin, Mi, -pi)
            if k == MOB_POLE:
                outr, outi = Mr, Mi
            else:
                outr = Mr * Mr - Mi * Mi
                outi = Mr * Mi + Mi * Mr
        elif k == MOBIUS:
            ar, ai, br, bi, cr, ci, dr, di = rec.p
            nr = (ar * zr - ai * zi) + br
            ni = (ar * zi + ai * zr) + bi
            dr_ = (cr * zr - ci * zi) + dr
            di_ = (cr * zi + ci * zr) + di
            outr, outi = _cdiv(nr, ni, dr_, di_)
            if cr != 0.0 or ci != 0.0:
                qr, qi = _cdiv(ar, ai, cr, ci)
                outr = np.where(fin, outr, qr)
                outi = np.where(fin, outi, qi)
            else:
                outinf |= zinf
        else:
            raise ValueError(k)
    outr = np.where(mode == ZERO, 0.0, outr)
    outi = np.where(mode == ZERO, 0.0, outi)
    outinf = (outinf | (mode == INF)) & (mode != ZERO)
    outr = np.where(outinf, 0.0, outr)
    outi = np.where(outinf, 0.0, outi)
    return Pts(outr, outi, outinf)


def apply_chain(chain, P: Pts) -> Pts:
    """Apply a recorded chain with the principal branch (points off every cut)."""
    for rec in chain:
        P = apply_rec(rec, P)
    return P


# ---------------------------------------------------------------- Algorithm 1

def _zip_sequence(z: Pts, k: int, branch: float):
    """g_1, ..., g_k of the geodesic algorithm on z_0..z_k; returns (maps, images)."""
    idx = np.arange(k + 1)
    maps = []
    r = rec_sqrt_ratio(complex(z.re[0], z.im[0]), complex(z.re[1], z.im[1]))
    maps.append(r)
    mode = np.where(idx == 0, INF, np.where(idx == 1, ZERO, PRINCIPAL)).astype(np.int8)
    P = apply_rec(r, z, mode)
    for j in range(2, k + 1):
        xr, xi = float(P.re[j]), float(P.im[j])
        if P.inf[j] or not (xr > 0.0):
            raise OracleError("NUMERIC", f"zipper step {j}: xi not in the right half-plane")
        r = rec_open(xr, xi, branch)
        maps.append(r)
        mode = np.where(idx < j - 1, SIGN, np.where(idx == j - 1, BRANCH,
                        np.where(idx == j, ZERO, PRINCIPAL))).astype(np.int8)
        P = apply_rec(r, P, mode)
    return maps, P


def intermediate_form(z: Pts, k: int, branch: float):
    """Algorithm 1 on the arc points z_0..z_k (k >= 2) with branching +-i.

    Returns (maps g_1..g_{k+1}, images Z_0..Z_k) with Z_0 = inf, Z_k = 0 and
    Z_1..Z_{k-1} on the imaginary axis.  Other points (the rest of the loop, the
    auxiliary points, interior points) never meet a cut; they get the recorded
    maps with the principal branch via ``apply_chain``.
    """
    if k < 2:
        raise OracleError("SCHEDULE", "an arc needs k >= 2")
    assert len(z) == k + 1
    idx = np.arange(k + 1)
    maps, P = _zip_sequence(z, k, branch)
    if P.inf[0]:
        raise OracleError("NUMERIC", "Algorithm 1: z_0 still at infinity")
    r = rec_mob_pole(float(P.re[0]), float(P.im[0]))
    maps.append(r)
    mode = np.where(idx == 0, INF, np.where(idx == k, ZERO, PRINCIPAL)).astype(np.int8)
    P = apply_rec(r, P, mode)
    return maps, P


# ---------------------------------------------------------------- Algorithm 2

def weld_maps(A: Pts, B: Pts, k: int):
    """Alignment maps of Algorithm 2 from the intermediate forms A_0..A_k, B_0..B_k.

    Returns (h_{k-1}, ..., h_1, h_0) and the images of the arc points on each
    side (A_j and B_j coincide from their own h_j on).
    """
    X = A.copy()
    Y = B.copy()
    idx = np.arange(k + 1)
    hs = []
    for j in range(k - 1, 0, -1):
        r = rec_close(float(X.im[j]), float(Y.im[j]))
        hs.append(r)
        mode = np.where(idx < j, SIGN, np.where(idx == j, ZERO, PRINCIPAL)).astype(np.int8)
        X = apply_rec(r, X, mode)
        Y = apply_rec(r, Y, mode)
    if X.inf[0]:
        raise OracleError("NUMERIC", "Algorithm 2: the shared point is still at infinity")
    r = rec_pole_sq(float(X.re[0]), float(X.im[0]))
    hs.append(r)
    mode = np.where(idx == 0, INF, PRINCIPAL).astype(np.int8)
    X = apply_rec(r, X, mode)
    Y = apply_rec(r, Y, mode)
    return hs, X, Y


# ---------------------------------------------------------------- geodesic disk map

def geodesic_disk(z: Pts, center: Pts):
    """Geodesic algorithm (Sec. 3.4) on the whole boundary z_0..z_n, then onto the disk.

    g_1, g_2..g_n with branching +i, g_{n+1}(z) = (z / (1 - z/p))^2 onto the
    upper half-plane.  The paper does not name the half-plane-to-disk map;
    we take w -> (w - c)/(w - conj c), where c is the half-plane image of the
    component's interior reference point, so that point goes to 0 and z_0 goes
    to 1.  (A plain Cayley map would put the preimage of 0 next to the closing
    edge z_n z_0 and give that one edge half of the circle.)
    Returns (chain, boundary images).
    """
    n = len(z) - 1
    if n < 2:
        raise OracleError("TOPOLOGY", "boundary loop too short")
    idx = np.arange(n + 1)
    maps, P = _zip_sequence(z, n, 1.0)
    r = rec_pole_sq(float(P.re[0]), float(P.im[0]))
    maps.append(r)
    mode = np.where(idx == 0, INF, np.where(idx == n, ZERO, PRINCIPAL)).astype(np.int8)
    P = apply_rec(r, P, mode)
    c = apply_chain(maps, center)
    if c.inf[0] or not (c.im[0] > 0.0):
        raise OracleError("NUMERIC", "disk centre is not in the upper half-plane")
    r = rec_half_plane_to_disk(float(c.re[0]), float(c.im[0]))
    maps.append(r)
    P = apply_rec(r, P)
    return maps, P
