"""Pins for the oracle's whole pipeline (Algorithm 3) and its metrics (Section 5).

* planar unit disk -> the disk map must be a Mobius automorphism of the input;
  the fit residual is discretisation error and must shrink under refinement;
* round sphere -> the spherical map must be a Mobius image of the input
  (conformal automorphisms of the sphere), again shrinking under refinement;
* the small disk case: no flipped faces, boundary on the unit circle, interior
  inside, seams coincide, weld-map estimate close to the harmonic solution;
* cut robustness (Table "cut_edges" idea): one mesh, five cut families, disk
  maps equal up to a disk automorphism;
* angle distortion, folds and |mu| on hand-computed triangles.
"""
import math

import numpy as np
import pytest

from oracle.pipeline import pgcp, stereo_from_plane, stereo_from_inverted
from oracle.metrics import angle_distortion, fold_check, beltrami_abs
from paper_1903_12359_gb300 import meshgen


def _mobius_fit_residual(z, w):
    A = np.column_stack([z, np.ones_like(z), -w * z, -w])
    _, _, vh = np.linalg.svd(A, full_matrices=False)
    a, b, c, d = vh[-1].conj()
    return np.abs((a * z + b) / (c * z + d) - w).max()


def test_planar_disk_is_a_disk_automorphism():
    res = []
    for rings, sectors in [(10, 16), (20, 32), (40, 64)]:
        m = meshgen.polar_disk_mesh(rings=rings, sectors=sectors, jitter=0.0, seed=0)
        m.V[:, 2] = 0.0
        r = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk")
        z = m.V[:, 0] + 1j * m.V[:, 1]
        w = r.out[:, 0] + 1j * r.out[:, 1]
        res.append(_mobius_fit_residual(z, w))
    assert res[-1] < 5e-3
    assert res[0] / res[1] > 2.5 and res[1] / res[2] > 2.5


def _sphere_to_plane(p):
    return (p[:, 0] - 1j * p[:, 1]) / (1.0 - p[:, 2])


@pytest.mark.slow
def test_round_sphere_is_a_mobius_image():
    res = []
    for sd in (4, 5, 6):     # subdivision 3 (642 vertices) is still pre-asymptotic
        m = meshgen.icosphere_sh_mesh(subdiv=sd, seed=0, amp=0.0)
        r = pgcp(m.V, m.F, face_labels=m.face_labels, variant="sphere")
        assert np.abs(np.linalg.norm(r.out, axis=1) - 1).max() < 1e-14
        P = m.V / np.linalg.norm(m.V, axis=1, keepdims=True)
        with np.errstate(divide="ignore", invalid="ignore"):
            z, w = _sphere_to_plane(P), _sphere_to_plane(r.out)
        ok = (np.abs(z) < 5) & (np.abs(w) < 5)
        res.append(_mobius_fit_residual(z[ok], w[ok]))
    assert res[-1] < 1e-3
    assert res[0] / res[1] > 2.5 and res[1] / res[2] > 2.5


def test_small_disk_case():
    m = meshgen.polar_disk_mesh()
    r = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk", map_interior=True)
    assert r.part.K == 2 and [(w.piece, w.k) for w in r.welds] == [(1, 80)]
    assert r.seam_mismatch == 0.0
    fc = fold_check(m.V, m.F, r.out)
    assert fc["flips"] == 0 and fc["folds"] == 0
    rad = np.hypot(r.out[:, 0], r.out[:, 1])
    loop = r.welds[-1].new_loop
    assert np.abs(rad[loop] - 1).max() < 1e-14
    inner = np.setdiff1d(np.arange(m.nv), loop)
    assert rad[inner].max() < 1
    st = angle_distortion(m.V, m.F, r.out)
    assert st["mean"] < 1.5
    for i in range(2):                       # the weld map is nearly harmonic already
        assert np.nanmax(np.abs(r.welded[i] - r.final[i])) < 5e-3
    rf = pgcp(m.V, m.F, face_labels=m.face_labels, variant="free")
    assert fold_check(m.V, m.F, rf.out)["flips"] == 0
    assert angle_distortion(m.V, m.F, rf.out)["mean"] < st["mean"]


@pytest.mark.slow
def test_cut_robustness_disk_maps_agree_up_to_automorphism():
    """Table "cut_edges" idea: one mesh, several cut families.  The disk map of a
    simply-connected surface is unique up to a disk automorphism, so the
    results of different cuts must be Mobius images of each other up to
    discretisation error (which shrinks under refinement)."""
    worst = []
    for N in (3000, 12000):
        m = meshgen.heightfield_disk_mesh(N, seed=7, nx=4, ny=2)
        c = m.V[m.F, :2].mean(axis=1)
        fams = [(np.array([-0.45, 0.0, 0.45]), np.array([0.0])), (np.array([0.0]), np.array([])),
                (np.array([]), np.array([0.0])), (np.array([-0.45, 0.45]), np.array([])),
                (np.array([0.0]), np.array([0.0]))]
        outs = []
        for cx, cy in fams:
            lab = np.searchsorted(cx, c[:, 0]) + (len(cx) + 1) * np.searchsorted(cy, c[:, 1])
            r = pgcp(m.V, m.F, face_labels=lab, variant="disk")
            outs.append(r.out[:, 0] + 1j * r.out[:, 1])
        worst.append(max(_mobius_fit_residual(outs[0], o) for o in outs[1:]))
    assert worst[0] < 1e-2 and worst[1] < 0.6 * worst[0]


def test_metrics_on_hand_triangles():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.0]])
    F = np.array([[0, 1, 2]])
    U = np.array([[0, 0], [2, 0], [0, 1.0]])
    st = angle_distortion(V, F, U)
    d = math.degrees(math.atan(2.0)) - 45.0      # angle at (0,1): 63.43 vs 45; at (2,0): 26.57 vs 45
    assert abs(st["max"] - d) < 1e-12 and abs(st["median"] - d) < 1e-12
    assert abs(st["mean"] - 2 * d / 3) < 1e-12
    assert abs(st["sd"] - math.sqrt(2 * d * d / 9)) < 1e-12
    # mu of the shear: f(x + iy) = 2x + iy -> f_z = 3/2, f_zbar = 1/2
    assert abs(beltrami_abs(V, F, U)[0] - 1.0 / 3.0) < 1e-14
    assert fold_check(V, F, U)["flips"] == 0
    assert fold_check(V, F, U[:, ::-1])["flips"] == 1
    assert angle_distortion(V, F, 3.0 * U[:, :] * 0 + 2.5 * V[:, :2])["max"] < 1e-12


def test_stereographic_charts_agree():
    z = np.array([0.3 + 0.2j, -4 + 1j, 1e-3 - 2e-3j])
    a = stereo_from_plane(z)
    b = stereo_from_inverted(1.0 / z)
    assert np.abs(a - b).max() < 1e-15
    assert np.abs(np.linalg.norm(a, axis=1) - 1).max() < 1e-15


def test_welded_map_is_invariant_to_each_piece_s_rotation_and_scale():
    """Section 4.3: the first map of Algorithm 1 on a piece depends only on
    ratios of its points, so multiplying a piece's local coordinates by a
    complex factor (rotation and scale, which keeps its reference point at 0)
    leaves the welded, disk and final maps unchanged up to rounding."""
    m = meshgen.heightfield_disk_mesh(3000, seed=9, nx=2, ny=2)
    r = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk")
    rng = np.random.default_rng(4)
    factors = [complex(*rng.uniform(0.3, 3.0, 2)) * np.exp(1j * rng.uniform(0, 2 * np.pi)) for _ in r.local]
    r2 = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk", local=[f * u for f, u in zip(factors, r.local)])
    assert r.part.K == 4 and len(r.welds) == 3
    assert np.abs(r2.out - r.out).max() < 1e-9
