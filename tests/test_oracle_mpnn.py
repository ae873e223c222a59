"""Pins of the FP64 message-passing network of the learned warm start
(oracle/mpnn.py): its gradient against central finite differences of its own
loss, the random-walk aggregation, and features that vanish where the weld-map
start is already discrete harmonic (linear maps on a planar mesh)."""
import numpy as np

from oracle import mpnn
from oracle.laplacian import cotan_laplacian
from paper_1903_12359_gb300 import meshgen


def _piece(rings=3, sectors=8, planar=False):
    m = meshgen.polar_disk_mesh(rings=rings, sectors=sectors, jitter=0.0)
    V = m.V.copy()
    if planar:
        V[:, 2] = 0.0
    L = cotan_laplacian(V, m.F)
    nv = V.shape[0]
    is_bnd = np.zeros(nv, dtype=bool)
    r = np.hypot(V[:, 0], V[:, 1])
    is_bnd[np.isclose(r, 1.0)] = True
    return V, L, is_bnd


def test_gradient_matches_finite_differences():
    V, L, is_bnd = _piece()
    rng = np.random.default_rng(3)
    u_w = rng.normal(size=(V.shape[0], 2))
    F, sigma = mpnn.features(L, is_bnd, u_w)
    P = mpnn.aggregation(L)
    theta = 0.5 * meshgen.he_normal(5, mpnn.param_shapes())
    theta[-16:] = rng.normal(size=16) * 0.1          # nonzero output bias
    target = rng.normal(size=(V.shape[0], 2))
    inner = ~is_bnd
    g = mpnn.gradient(theta, F, P, target, inner)
    assert g.size == mpnn.n_params() == 35152
    idx = rng.choice(theta.size, size=80, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mpnn.loss(tp, F, P, target, inner) - mpnn.loss(tm, F, P, target, inner)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_aggregation_is_a_random_walk():
    V, L, is_bnd = _piece(rings=5, sectors=12)
    P = mpnn.aggregation(L)
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-12)
    assert np.all(P.diagonal() == 0.0)


def test_features_vanish_for_linear_maps_on_planar_mesh():
    V, L, is_bnd = _piece(rings=5, sectors=12, planar=True)
    u = V[:, 0:2] @ np.array([[2.0, -1.0], [0.5, 3.0]]) + np.array([0.3, -0.7])
    F, sigma = mpnn.features(L, is_bnd, u)
    # z = sigma * F vanishes up to rounding (linear precision of the cotan Laplacian)
    assert np.abs(F[:, 0:2]).max() * sigma < 1e-12 * max(1.0, np.abs(u).max())
    assert np.array_equal(F[:, 2], is_bnd.astype(float)) and np.all(F[:, 3] == 1.0)
    # a harmonic-in-z perturbation of the interior is seen
    u2 = u.copy()
    u2[~is_bnd] += 1e-3
    F2, s2 = mpnn.features(L, is_bnd, u2)
    assert s2 > 0 and np.abs(F2[:, 0:2]).max() > 0.5


def test_zero_weights_give_the_output_bias():
    V, L, is_bnd = _piece()
    F, _ = mpnn.features(L, is_bnd, np.random.default_rng(0).normal(size=(V.shape[0], 2)))
    P = mpnn.aggregation(L)
    theta = np.zeros(mpnn.n_params())
    theta[-16:] = np.arange(16.0)
    out = mpnn.forward(theta, F, P)
    assert np.allclose(out, np.arange(16.0)[None, :])
