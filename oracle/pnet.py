"""FP64 oracle of the paper's own surrogate network (arXiv 2206.02937,
Sec. 3.2): three hidden layers of 9, 12 and 9 ReLU units and one sigmoid
output.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only the tests, the smoke
check and the CPU-baseline leg of the benchmark use it.

Inputs (Fig. 2a lists the two momenta, the two macro-particle weights and the
maximum probability P_max of the cell): nine features

    f = [sgnlog(u_i / s_u) / n_u, sgnlog(k_i / s_k) / n_k,      i = x, y, z
         ln(w_e) / 8, ln(w_g) / 8, ln(P_max) / 8],

sgnlog(z) = sign(z) log(1 + |z|), with w the macro-particle weight over the
cell volume and P_max = 2 n dt the cell's probability bound (sigma_T c = 1);
target r = sigma_KN v / (2 sigma_T), as for the larger network.  The loss is
the (weighted) mean absolute error; the ReLU subgradient at 0 is 0.

Parameter vector (float64, length 337), layer by layer, W stored (out, in):
    W0 (9 x 9), b0 (9), W1 (12 x 9), b1 (12), W2 (9 x 12), b2 (9), W3 (1 x 9), b3 (1)
"""
from __future__ import annotations

import numpy as np

from oracle.mlp import sgnlog

SHAPES = [(9, 9), (12, 9), (9, 12), (1, 9)]
N_PARAMS = sum(o * i + o for o, i in SHAPES)


def unpack(theta: np.ndarray):
    out, at = [], 0
    for o, i in SHAPES:
        W = theta[at:at + o * i].reshape(o, i)
        at += o * i
        b = theta[at:at + o]
        at += o
        out.append((W, b))
    return out


def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(N_PARAMS)
    for W, b in unpack(theta):
        lim = np.sqrt(6.0 / (W.shape[0] + W.shape[1]))
        W[...] = rng.uniform(-lim, lim, W.shape)
    return theta


def features(u, k, w_e, w_g, p_max, scales=(1.0, 7.0, 1e-4, 10.0)) -> np.ndarray:
    """(9, n) inputs from (3, n) momenta and per-pair (or scalar) weights and
    P_max."""
    u = np.asarray(u, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    n = u.shape[1]
    s_u, n_u, s_k, n_k = scales
    f = np.zeros((9, n))
    f[0:3] = sgnlog(u / s_u) / n_u
    f[3:6] = sgnlog(k / s_k) / n_k
    f[6] = np.log(np.broadcast_to(np.asarray(w_e, dtype=np.float64), (n,))) / 8.0
    f[7] = np.log(np.broadcast_to(np.asarray(w_g, dtype=np.float64), (n,))) / 8.0
    f[8] = np.log(np.broadcast_to(np.asarray(p_max, dtype=np.float64), (n,))) / 8.0
    return f


def forward(theta: np.ndarray, f: np.ndarray):
    layers = unpack(theta)
    h = np.asarray(f, dtype=np.float64)
    cache = [h]
    for W, b in layers[:-1]:
        z = W @ h + b[:, None]
        h = np.maximum(z, 0.0)
        cache += [z, h]
    W, b = layers[-1]
    z = W @ h + b[:, None]
    y = 1.0 / (1.0 + np.exp(-z[0]))
    return y, cache


def backward(theta: np.ndarray, f: np.ndarray, y: np.ndarray, w=None):
    """Weighted MAE and its gradient (same layout as theta)."""
    y_pred, cache = forward(theta, f)
    n = y.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    loss = float(np.sum(w * np.abs(y_pred - y)) / np.sum(w))
    grad = np.zeros_like(theta)
    gl = unpack(grad)
    layers = unpack(theta)
    dz = (w * np.sign(y_pred - y) / np.sum(w) * y_pred * (1.0 - y_pred))[None, :]
    gl[-1][0][...] = dz @ cache[-1].T
    gl[-1][1][...] = dz.sum(axis=1)
    dh = layers[-1][0].T @ dz
    for li in range(len(SHAPES) - 2, -1, -1):
        z = cache[1 + 2 * li]
        dz = dh * (z > 0.0)
        gl[li][0][...] = dz @ cache[2 * li].T
        gl[li][1][...] = dz.sum(axis=1)
        dh = layers[li][0].T @ dz
    return loss, grad
