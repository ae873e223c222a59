"""Pins for the oracle's area distortion and Mobius area step (Section 6.2).

* hand triangles: d_area from the definition, worked by hand;
* similarities leave d_area unchanged, and a similar copy of a planar mesh
  has d_area = 0 everywhere;
* the families: f_{-alpha} o f_alpha = id and |f_alpha| = 1 on the unit
  circle (disk); f_q o f_p = f_{p+q} (free);
* Nelder-Mead finds the minimum of a quadratic;
* a planar disk mapped by a known family member is mapped back: the step
  finds the inverse parameter and d_area ~ 0;
* on the small disk case the step does not increase mean |d_area|.
"""
import math

import numpy as np

from oracle import area as AR
from oracle.pipeline import pgcp
from paper_1903_12359_gb300 import meshgen


def test_hand_triangles():
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0.0]])
    F = np.array([[0, 1, 2], [0, 2, 3]])
    # surface areas 1/2 and 1/2; parameter areas 1 ((0,0),(2,0),(2,1)) and 1/2 ((0,0),(2,1),(0,1/2))
    U = np.array([[0, 0], [2, 0], [2, 1], [0, 0.5]])
    d = AR.area_distortion(V, F, U)
    assert abs(d[0] - math.log((1.0 / 1.5) / 0.5)) < 1e-14
    assert abs(d[1] - math.log((0.5 / 1.5) / 0.5)) < 1e-14


def test_similarities_do_not_change_area_distortion():
    m = meshgen.polar_disk_mesh(rings=8, sectors=16, seed=3)
    U = m.V[:, :2] * np.array([1.0, 0.7]) + 0.1 * m.V[:, :2] ** 2   # some planar map
    d0 = AR.area_distortion(m.V, m.F, U)
    z = U[:, 0] + 1j * U[:, 1]
    w = (2.5 - 1.5j) * z + (0.3 + 4j)
    d1 = AR.area_distortion(m.V, m.F, np.stack([w.real, w.imag], axis=1))
    assert np.abs(d0 - d1).max() < 1e-12
    flat = m.V.copy()
    flat[:, 2] = 0.0
    w = (0.5 + 0.5j) * (flat[:, 0] + 1j * flat[:, 1]) - 2.0
    assert np.abs(AR.area_distortion(flat, m.F, np.stack([w.real, w.imag], axis=1))).max() < 1e-12


def test_families():
    rng = np.random.default_rng(0)
    z = rng.normal(size=50) + 1j * rng.normal(size=50)
    a = 0.3 - 0.45j
    assert np.abs(AR.mobius("disk", -a, AR.mobius("disk", a, z)) - z).max() < 1e-12
    t = np.exp(1j * np.linspace(0, 2 * np.pi, 17))
    assert np.abs(np.abs(AR.mobius("disk", a, t)) - 1.0).max() < 1e-14
    p, q = 0.2 + 0.1j, -0.05 + 0.3j
    assert np.abs(AR.mobius("free", q, AR.mobius("free", p, z)) - AR.mobius("free", p + q, z)).max() < 1e-12


def test_nelder_mead_on_a_quadratic():
    x, f, n = AR.nelder_mead(lambda x: (x[0] - 1.0) ** 2 + 2.0 * (x[1] + 0.5) ** 2 + 3.0, [0.0, 0.0])
    assert np.abs(x - [1.0, -0.5]).max() < 1e-5 and abs(f - 3.0) < 1e-10 and n < 500


def _flat_disk():
    m = meshgen.polar_disk_mesh(rings=12, sectors=24, seed=1)
    flat = m.V.copy()
    flat[:, 2] = 0.0
    return m, flat


def test_step_undoes_a_known_automorphism_of_a_planar_disk():
    m, flat = _flat_disk()
    a0 = 0.35 + 0.2j
    w = AR.mobius("disk", a0, flat[:, 0] + 1j * flat[:, 1])
    U = np.stack([w.real, w.imag], axis=1)
    p, before, after, evals, W = AR.area_step(flat, m.F, U, "disk")
    assert before > 0.1 and after < 1e-6, (before, after)
    assert abs(p + a0) < 1e-6, p
    assert np.abs(W - flat[:, :2]).max() < 1e-5


def test_step_undoes_a_known_free_mobius_map():
    m, flat = _flat_disk()
    q0 = 0.25 - 0.15j                                   # pole 1/q0 outside the unit disk
    w = AR.mobius("free", q0, flat[:, 0] + 1j * flat[:, 1])
    U = np.stack([w.real, w.imag], axis=1)
    p, before, after, evals, W = AR.area_step(flat, m.F, U, "free")
    assert before > 0.05 and after < 1e-6, (before, after)
    assert abs(p + q0) < 1e-6, p


def test_step_on_the_small_disk_case():
    m = meshgen.polar_disk_mesh()
    r = pgcp(m.V, m.F, face_labels=m.face_labels, variant="disk")
    p, before, after, evals, W = AR.area_step(m.V, m.F, r.out, "disk")
    assert abs(p) < 1.0 and after <= before
    assert abs(before - np.abs(AR.area_distortion(m.V, m.F, r.out)).mean()) < 1e-14
    assert np.abs(np.hypot(W[:, 0], W[:, 1]).max() - 1.0) < 1e-12   # still the unit disk


def test_ball_automorphisms():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(40, 3))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    a = np.array([0.3, -0.2, 0.45])
    Y = AR.ball_automorphism(a, X)
    assert np.abs(np.linalg.norm(Y, axis=1) - 1.0).max() < 1e-14          # keeps the sphere
    assert np.abs(AR.ball_automorphism(np.zeros(3), X) - X).max() == 0.0   # T_0 = id
    assert np.abs(AR.ball_automorphism(a, a[None, :])).max() < 1e-15      # T_a(a) = 0
    assert np.abs(AR.ball_automorphism(a, np.zeros((1, 3))) + a).max() < 1e-15   # T_a(0) = -a
    Z = AR.ball_automorphism(-a, Y)                 # T_{-a} o T_a fixes 0: a rotation
    assert np.abs(Z @ Z.T - X @ X.T).max() < 1e-12


def test_step_undoes_a_known_sphere_automorphism():
    m = meshgen.icosphere_sh_mesh(subdiv=3, seed=0, amp=0.0)
    S = m.V / np.linalg.norm(m.V, axis=1, keepdims=True)
    a0 = np.array([0.25, 0.1, -0.3])
    X = AR.ball_automorphism(a0, S)
    a, before, after, evals, Y = AR.area_step(m.V, m.F, X, "sphere")
    assert before > 0.1 and after < 1e-6, (before, after)
    assert np.abs(a + a0).max() < 1e-5, a
    idx = np.arange(0, m.nv, 7)
    assert np.abs(Y[idx] @ Y[idx].T - S[idx] @ S[idx].T).max() < 1e-5   # a rotation of the input
