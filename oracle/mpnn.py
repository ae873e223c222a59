"""Learned warm start: the message-passing network, in FP64 (test infrastructure).

Not in the paper: a warm start for the final Laplace solve (Sec. 4.5) that the
plain method then verifies.  Definitions (the CUDA library computes the same
network in BF16 with FP32 accumulation):

Features of row i of a piece, from the weld-map start u_w and the piece's
positive semidefinite cotan Laplacian L with diagonal d:
    z_i   = -(1/d_i) sum_j L_ij u_w,j   on interior rows, 0 on boundary rows
    sigma = sqrt(mean over the piece's interior rows of |z_i|^2)   (1 if 0)
    F_i   = [z_i.x / sigma, z_i.y / sigma, boundary flag, 1, 0 x 12]   (16 wide)
Aggregation P = D^-1 W, with W_ij = -L_ij off the diagonal (random walk).
Network (width 64, 4 message-passing layers):
    X_0     = relu(F W_in + b_in)
    X_{l+1} = relu([X_l | P X_l] W_l + b_l),     l = 0..3   (W_l is 128 x 64)
    out     = X_4 W_out + b_out                   (W_out is 64 x 16; columns 0, 1 used)
Prediction: u_0 = u_w + sigma * out[:, 0:2] on interior rows.
Training target: t_i = (u*_i - u_w,i) / sigma on interior rows, where u* is
the solved final map.  Loss = (1 / n_interior) sum_interior |out_i[0:2] - t_i|^2.

Parameters are one flat vector: W_in (16 x 64), b_in (64), then for each layer
W_l (128 x 64), b_l (64), then W_out (64 x 16), b_out (16); matrices row-major
with rows = inputs.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import csr_matrix, diags

F_IN, WIDTH, LAYERS, F_OUT = 16, 64, 4, 16


def param_shapes():
    s = [(F_IN, WIDTH), (WIDTH,)]
    for _ in range(LAYERS):
        s += [(2 * WIDTH, WIDTH), (WIDTH,)]
    s += [(WIDTH, F_OUT), (F_OUT,)]
    return s


def n_params() -> int:
    return int(sum(np.prod(x) for x in param_shapes()))


def unpack(theta: np.ndarray):
    out, o = [], 0
    for shp in param_shapes():
        k = int(np.prod(shp))
        out.append(theta[o:o + k].reshape(shp))
        o += k
    return out


def features(L: csr_matrix, is_bnd: np.ndarray, u_w: np.ndarray):
    """(F [n x 16], sigma) for one piece; u_w complex or [n, 2]."""
    U = np.column_stack([u_w.real, u_w.imag]) if np.iscomplexobj(u_w) else np.asarray(u_w, dtype=np.float64)
    d = L.diagonal()
    z = -(L @ U) / d[:, None]
    z[is_bnd] = 0.0
    inner = ~is_bnd
    ms = float(np.mean(np.sum(z[inner] ** 2, axis=1))) if inner.any() else 0.0
    sigma = np.sqrt(ms) if ms > 0 else 1.0
    F = np.zeros((L.shape[0], F_IN))
    F[:, 0:2] = z / sigma
    F[:, 2] = is_bnd.astype(np.float64)
    F[:, 3] = 1.0
    return F, sigma


def aggregation(L: csr_matrix) -> csr_matrix:
    d = L.diagonal()
    W = -(L - diags(d))
    return (diags(1.0 / d) @ W).tocsr()


def forward(theta, F, P, keep=False):
    p = unpack(theta)
    Win, bin_ = p[0], p[1]
    X = np.maximum(F @ Win + bin_, 0.0)
    cache = [(F, None, X)]
    for l in range(LAYERS):
        W, b = p[2 + 2 * l], p[3 + 2 * l]
        A = np.hstack([X, P @ X])
        X = np.maximum(A @ W + b, 0.0)
        cache.append((A, None, X))
    out = X @ p[-2] + p[-1]
    return (out, cache) if keep else out


def loss(theta, F, P, target, inner):
    out = forward(theta, F, P)
    r = out[inner, 0:2] - target[inner]
    return float(np.sum(r * r) / max(int(inner.sum()), 1))


def gradient(theta, F, P, target, inner):
    """d loss / d theta by reverse-mode differentiation of forward()."""
    p = unpack(theta)
    out, cache = forward(theta, F, P, keep=True)
    n = max(int(inner.sum()), 1)
    dout = np.zeros_like(out)
    dout[inner, 0:2] = 2.0 * (out[inner, 0:2] - target[inner]) / n
    grads = [None] * len(p)
    X4 = cache[-1][2]
    grads[-2] = X4.T @ dout
    grads[-1] = dout.sum(axis=0)
    dX = dout @ p[-2].T
    for l in range(LAYERS - 1, -1, -1):
        A, _, Xn = cache[l + 1]
        dZ = dX * (Xn > 0)
        grads[2 + 2 * l] = A.T @ dZ
        grads[3 + 2 * l] = dZ.sum(axis=0)
        dA = dZ @ p[2 + 2 * l].T
        dX = dA[:, :WIDTH] + P.T @ dA[:, WIDTH:]
    X0 = cache[0][2]
    dZ = dX * (X0 > 0)
    grads[0] = F.T @ dZ
    grads[1] = dZ.sum(axis=0)
    return np.concatenate([g.reshape(-1) for g in grads])
