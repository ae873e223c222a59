"""Pins for the oracle's elementary maps, Algorithm 1, Algorithm 2 and the
geodesic disk map (Sections 3.2, 3.4, 4.3, 4.4.1).

Checked against: numpy / Python complex arithmetic for the scalar kernels, the
three-point properties the paper states for each Mobius map, cross-ratio
invariance, a 40-digit mpmath evaluation of Algorithm 1, the intermediate-form
shape Algorithm 1 promises, and convergence of the geodesic map of a circle to
the exact Riemann map (a rotation).
"""
import math

import numpy as np
import pytest

from oracle import welding as W
from oracle.mesh import partition, weld_schedule
from oracle.dncp import dncp
from paper_1903_12359_gb300 import meshgen

rng = np.random.default_rng(1234)


def _pts(z):
    return W.Pts.from_complex(np.atleast_1d(z))


def _apply(rec, z):
    return W.apply_rec(rec, _pts(z))


def test_scalar_kernels():
    x = rng.normal(size=2000) * np.exp(rng.uniform(-20, 20, size=2000))
    y = rng.normal(size=2000) * np.exp(rng.uniform(-20, 20, size=2000))
    x[:10] = -np.abs(x[:10]); y[:5] = 0.0; y[5:10] = -0.0
    rr, ri = W._csqrt(x, y)
    zc = np.empty(x.size, dtype=complex)
    zc.real, zc.imag = x, y                 # keeps the sign of zero imaginary parts
    ref = np.sqrt(zc)
    assert np.all(rr >= 0)
    assert np.all(np.abs((rr + 1j * ri) - ref) <= 4e-16 * np.abs(ref))
    assert np.array_equal(np.signbit(ri[5:10]), np.ones(5, dtype=bool))   # -0 keeps the lower side
    br, bi = rng.normal(size=2000), rng.normal(size=2000)
    qr, qi = W._cdiv(x, y, br, bi)
    q = (x + 1j * y) / (br + 1j * bi)
    assert np.all(np.abs((qr + 1j * qi) - q) <= 1e-15 * np.abs(q))
    h = W._hypot(x, y)
    assert np.all(np.abs(h - np.hypot(x, y)) <= 4.5e-16 * np.hypot(x, y))


def _cross_ratio(a, b, c, d):
    return (a - c) * (b - d) / ((a - d) * (b - c))


def test_mobius_three_point_properties():
    for _ in range(20):
        xi = complex(rng.uniform(0.1, 3), rng.normal())
        rec = W.rec_open(xi.real, xi.imag, 1.0)
        cr, ci = rec.p
        _, _, L0r, L0i = W._mob_open(cr, ci, 0.0, 0.0)
        _, _, L1r, L1i = W._mob_open(cr, ci, xi.real, xi.imag)
        rho = 1j * abs(xi) ** 2 / xi.imag
        Dr, Di, _, _ = W._mob_open(cr, ci, rho.real, rho.imag)
        assert abs(complex(L0r, L0i)) == 0.0                      # L(0) = 0
        assert abs(complex(L1r, L1i) - 1.0) < 1e-14               # L(xi) = 1
        assert abs(complex(Dr, Di)) < 1e-14 * abs(rho) * abs(ci)  # L(rho) = inf
        a, b = rng.uniform(0.1, 5), -rng.uniform(0.1, 5)
        if rng.uniform() < 0.5:                                    # the wrapped order 0 < a < b
            a, b = sorted([rng.uniform(0.1, 5), rng.uniform(5, 9)])
        rec = W.rec_close(a, b)
        c1, c2 = rec.p
        T = lambda z: complex(*[float(t) for t in W._mob_close(c1, c2, z.real, z.imag)[2:]])
        assert abs(T(1j * a) - 1j) < 1e-13 and abs(T(1j * b) + 1j) < 1e-13 and T(0j) == 0
        z = complex(rng.uniform(0, 3), rng.normal())
        assert T(z).real > 0                                       # keeps the right half-plane
    p = rng.normal(size=3) + 1j * rng.normal(size=3)
    r = W.rec_normalize(p[0], p[1], p[2])
    out = _apply(r, p)
    assert abs(out.complex()[0] + 1) < 1e-12 and abs(out.complex()[1] - 1) < 1e-12
    near = _apply(r, np.array([p[2] + 1e-9])).complex()[0]     # p3 is the pole
    assert abs(near) > 1e6
    q = complex(rng.normal(), rng.normal())
    r = W.rec_sphere_frame(p[0], p[1], q, invert=False)
    out = _apply(r, np.array([p[0], q]))
    assert abs(out.complex()[0]) < 1e-13 and abs(out.complex()[1] - 1) < 1e-13
    c = complex(rng.normal(), abs(rng.normal()) + 0.1)
    r = W.rec_half_plane_to_disk(c.real, c.imag)
    out = _apply(r, np.array([c, 3.7, -12.0]))
    assert abs(out.complex()[0]) < 1e-15
    assert np.allclose(np.abs(out.complex()[1:]), 1.0, atol=1e-15)
    assert abs(W.apply_rec(r, W.Pts([0.0], [0.0], [True])).complex()[0] - 1) < 1e-15


def test_cross_ratio_invariance():
    z = rng.normal(size=4) + 1j * rng.normal(size=4)
    cr0 = _cross_ratio(*z)
    recs = [W.rec_normalize(*(rng.normal(size=3) + 1j * rng.normal(size=3))),
            W.rec_sphere_frame(*(rng.normal(size=3) + 1j * rng.normal(size=3)), invert=True),
            W.rec_half_plane_to_disk(0.3, 0.7),
            W.rec_mob_pole(0.2, 1.3)]
    for r in recs:
        w = _apply(r, z).complex()
        assert abs(_cross_ratio(*w) - cr0) < 1e-12 * abs(cr0)
    xi = complex(0.7, 0.4)
    cr, ci = W.rec_open(xi.real, xi.imag, 1.0).p
    L = np.array([complex(*[float(t) for t in W._mob_open(cr, ci, v.real, v.imag)[2:]]) for v in z])
    assert abs(_cross_ratio(*L) - cr0) < 1e-12 * abs(cr0)


def _c1_first_weld_arc():
    m = meshgen.polar_disk_mesh()
    P = partition(m.V, m.F, face_labels=m.face_labels)
    w = weld_schedule(P, False)[0]
    X = m.V[P.verts[0]]
    ll = np.searchsorted(P.verts[0], P.loops[0])
    u, _ = dncp(X, P.local_F[0], ll)
    pos = {g: i for i, g in enumerate(P.verts[0].tolist())}
    z = np.array([u[pos[g]] for g in w.a.tolist()])
    return z, w.k


@pytest.mark.parametrize("branch", [1.0, -1.0])
def test_intermediate_form_shape(branch):
    z, k = _c1_first_weld_arc()
    maps, A = W.intermediate_form(_pts(z[:k + 1]), k, branch)
    assert len(maps) == k + 1
    assert A.inf[0] and not A.inf[1:].any()
    assert A.re[k] == 0.0 and A.im[k] == 0.0
    Z = A.complex()[1:k]
    assert np.all(np.abs(Z.real) <= 1e-12 * np.abs(Z))
    assert np.all(np.sign(Z.imag) == branch)
    assert np.all(np.diff(np.abs(Z.imag)) < 0)                    # ordered from infinity down to 0
    rest = W.apply_chain(maps, _pts(z[k + 1:]))                   # the other loop points
    assert np.all(rest.re > 0)


def test_intermediate_form_matches_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    z, k = _c1_first_weld_arc()
    k = 40
    zz = z[:k + 1]
    _, A = W.intermediate_form(_pts(zz), k, 1.0)
    Z = [mp.mpc(v.real, v.imag) for v in zz]
    P = [mp.inf, mp.mpc(0)] + [mp.sqrt((Z[l] - Z[1]) / (Z[l] - Z[0])) for l in range(2, k + 1)]
    for j in range(2, k + 1):
        xi = P[j]
        s = abs(xi) ** 2
        cr, ci = xi.real / s, xi.imag / s
        Q = []
        for l, x in enumerate(P):
            L = mp.mpc(0, -cr / ci) if x == mp.inf else cr * x / (1 + ci * x * 1j)
            r = mp.sqrt(L * L - 1)
            if l < j - 1 and r.imag * L.imag < 0:
                r = -r
            if l == j - 1:
                r = mp.mpc(0, 1)
            if l == j:
                r = mp.mpc(0)
            Q.append(r)
        P = Q
    ref = [P[l] / (1 - P[l] / P[0]) for l in range(1, k)]
    got = A.complex()[1:k]
    err = max(float(abs(complex(r) - g) / abs(r)) for r, g in zip(ref, got))
    assert err < 1e-12


def test_weld_maps_pair_up_the_arc():
    z, k = _c1_first_weld_arc()
    m = meshgen.polar_disk_mesh()
    P = partition(m.V, m.F, face_labels=m.face_labels)
    w = weld_schedule(P, False)[0]
    X1 = m.V[P.verts[1]]
    ll1 = np.searchsorted(P.verts[1], P.loops[1])
    u1, _ = dncp(X1, P.local_F[1], ll1)
    pos = {g: i for i, g in enumerate(P.verts[1].tolist())}
    zb = np.array([u1[pos[g]] for g in w.b.tolist()])
    gA, A = W.intermediate_form(_pts(z[:k + 1]), k, 1.0)
    gB, B = W.intermediate_form(_pts(zb[:k + 1]), k, -1.0)
    hs, X, Y = W.weld_maps(A, B, k)
    assert len(hs) == k
    # Algorithm 2's postcondition: after the whole chain the two images of every
    # shared arc point coincide, a~_j = b~_j for 1 <= j <= k (a_0 = b_0 goes to
    # infinity on both sides), to 1e-10 relative
    assert X.inf[0] and Y.inf[0]
    xa, yb = X.complex()[1:k + 1], Y.complex()[1:k + 1]
    rel = np.abs(xa - yb) / np.maximum(np.abs(xa), 1.0)
    assert rel.max() < 1e-10, rel.max()
    # each h_j closes its own pair: recomputed by the chain without the index
    # rule, alpha_j and beta_j land at 0 up to the rounding of that evaluation
    for j in (k - 1, k // 2, 1):
        a = W.apply_chain(hs[:k - 1 - j], A.take([j]))
        b = W.apply_chain(hs[:k - 1 - j], B.take([j]))
        ha = W.apply_rec(hs[k - 1 - j], a).complex()[0]
        hb = W.apply_rec(hs[k - 1 - j], b).complex()[0]
        assert abs(ha) < 1e-6 and abs(hb) < 1e-6


def test_weld_puts_the_two_pieces_on_opposite_sides_of_the_seam():
    """After the weld of the small disk case (two pieces, Algorithm 2 plus the
    normalisation), every face of both pieces keeps a positive signed area
    (interior points mapped through their side's chain) and the faces together
    cover the region bounded by the image of the outer loop exactly once: the
    sum of the face areas equals that loop's polygon area.  If the two pieces
    landed on the same side of the seam their images would overlap and the sum
    would exceed the polygon area."""
    m = meshgen.polar_disk_mesh()
    from oracle.pipeline import pgcp as o_pgcp
    res = o_pgcp(m.V, m.F, face_labels=m.face_labels, variant="free", map_interior=True)
    P = res.part
    total = 0.0
    for i in range(P.K):
        z = res.welded[i]
        assert not res.welded_inf[i].any()
        Fl = P.local_F[i]
        a, b, c = z[Fl[:, 0]], z[Fl[:, 1]], z[Fl[:, 2]]
        area = 0.5 * ((b - a).real * (c - a).imag - (b - a).imag * (c - a).real)
        assert area.min() > 0.0
        total += float(area.sum())
    outer = res.welds[-1].new_loop
    pos = {}
    for i in range(P.K):
        for li, g in enumerate(P.verts[i].tolist()):
            pos.setdefault(g, (i, li))
    w = np.array([res.welded[pos[g][0]][pos[g][1]] for g in outer.tolist()])
    poly = 0.5 * float(np.sum(w.real * np.roll(w.imag, -1) - w.imag * np.roll(w.real, -1)))
    assert poly > 0.0
    assert abs(total - poly) < 1e-9 * poly, (total, poly)


def test_geodesic_disk_converges_to_rotation_on_a_circle():
    errs = []
    c = 0.3 + 0.1j
    for n in (32, 64, 128, 256):
        th = 2 * np.pi * np.arange(n) / n + 0.3 * np.sin(np.arange(n)) * 2 * np.pi / n
        z = 2.0 * np.exp(1j * th) + c
        chain, img = W.geodesic_disk(_pts(z), _pts(c))
        w = img.complex()
        assert np.abs(np.abs(w) - 1).max() < 1e-14
        rot = w / ((z - c) / 2)
        errs.append(np.abs(rot - rot.mean()).max())
        inner = W.apply_chain(chain, _pts(c + np.array([0.5, -0.7j])))
        assert np.all(np.abs(inner.complex()) < 1)
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.5)                                   # second order
