"""FP64 oracle of the surrogate network (arXiv 2206.02937, Sec. 2 and 3.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only the tests, the smoke
check and the CPU-baseline leg of the benchmark use it.

The paper's network maps the photon and lepton momenta (units of m_e c) to a
probability y' in [0, 1] with fully connected layers, hidden activations and a
sigmoid output (Sec. 3.2); it is trained with the mean absolute error and the
Adam optimizer at learning rate 1e-3 (Sec. 3.2, Kingma and Ba 2014).  The
configuration built here is 4 hidden layers of 64 SiLU units (the paper's own
9-12-9 ReLU network is a later variant), inputs

    f = [sgnlog(u_i / s_u) / n_u, sgnlog(k_i / s_k) / n_k],  i = x, y, z,
    sgnlog(z) = sign(z) log(1 + |z|),

target r = sigma_KN v / (2 sigma_T) (the probability normalised by the cell
maximum P_max = 2 sigma_T c dt max w of Sec. 3.2).

Parameter vector layout (float64, length 12993), layer by layer:
    W0 (64 x 6), b0 (64), W1 (64 x 64), b1, W2, b2, W3, b3, W4 (1 x 64), b4 (1)
with W stored (out, in), row-major.  The library uses the same vector.
"""
from __future__ import annotations

import numpy as np

N_IN, WIDTH, DEPTH = 6, 64, 4
FEATURE_SCALES = dict(s_u=1.0, n_u=7.0, s_k=1e-4, n_k=10.0)


def layer_shapes():
    shapes = [(WIDTH, N_IN)] + [(WIDTH, WIDTH)] * (DEPTH - 1) + [(1, WIDTH)]
    return shapes


def n_params() -> int:
    return sum(o * i + o for o, i in layer_shapes())


def unpack(theta: np.ndarray):
    """[(W, b), ...] views into the flat parameter vector."""
    out, at = [], 0
    for o, i in layer_shapes():
        W = theta[at:at + o * i].reshape(o, i)
        at += o * i
        b = theta[at:at + o]
        at += o
        out.append((W, b))
    assert at == theta.shape[0]
    return out


def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases (Keras' default initialisation)."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(n_params())
    for W, b in unpack(theta):
        lim = np.sqrt(6.0 / (W.shape[0] + W.shape[1]))
        W[...] = rng.uniform(-lim, lim, W.shape)
    return theta


def sgnlog(z):
    return np.sign(z) * np.log1p(np.abs(z))


def pair_invariants(u: np.ndarray, k: np.ndarray):
    """(x, v) per pair from (3, n) momenta, in FP64: gamma = sqrt(1 + |u|^2),
    eps = |k|, x = gamma eps - u.k (the photon energy in the electron rest
    frame), v = x / (gamma eps) = 1 - beta cos psi (1 for eps = 0)."""
    u = np.asarray(u, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    gamma = np.sqrt(1.0 + (u * u).sum(0))
    eps = np.sqrt((k * k).sum(0))
    x = gamma * eps - (u * k).sum(0)
    ge = gamma * eps
    v = np.where(ge > 0, x / np.where(ge > 0, ge, 1.0), 1.0)
    return x, v


def features(u: np.ndarray, k: np.ndarray, scales=FEATURE_SCALES, mode: str = "momenta") -> np.ndarray:
    """(6, n) network inputs from (3, n) momenta.  mode "momenta": the six
    sgnlog-scaled components; mode "invariants": [ln(x)/8, ln(v)/8, 0, 0, 0, 0]
    (x, v floored at 1e-30)."""
    u = np.asarray(u, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    if mode == "invariants":
        x, v = pair_invariants(u, k)
        f = np.zeros((6, u.shape[1]))
        f[0] = np.log(np.maximum(x, 1e-30)) / 8.0
        f[1] = np.log(np.maximum(v, 1e-30)) / 8.0
        return f
    return np.concatenate([sgnlog(u / scales["s_u"]) / scales["n_u"],
                           sgnlog(k / scales["s_k"]) / scales["n_k"]])


def silu(z):
    return z / (1.0 + np.exp(-z))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(theta: np.ndarray, f: np.ndarray):
    """y' for (6, n) inputs f; returns (y', cache of pre-activations and activations)."""
    layers = unpack(theta)
    h = np.asarray(f, dtype=np.float64)
    cache = [h]
    for W, b in layers[:-1]:
        z = W @ h + b[:, None]
        h = silu(z)
        cache += [z, h]
    W, b = layers[-1]
    z = W @ h + b[:, None]
    y = sigmoid(z)[0]
    cache.append(z)
    return y, cache


def mae_loss(y_pred, y, w=None) -> float:
    """Weighted mean absolute error sum w |y' - y| / sum w (Sec. 3.2, MAE)."""
    w = np.ones_like(y) if w is None else w
    return float(np.sum(w * np.abs(y_pred - y)) / np.sum(w))


def backward(theta: np.ndarray, f: np.ndarray, y: np.ndarray, w=None):
    """Loss and its gradient w.r.t. theta (same layout).  The MAE subgradient
    at y' = y is taken as 0."""
    y_pred, cache = forward(theta, f)
    n = y.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    loss = float(np.sum(w * np.abs(y_pred - y)) / np.sum(w))
    grad = np.zeros_like(theta)
    gl = unpack(grad)
    layers = unpack(theta)
    # d loss / d y'
    dy = w * np.sign(y_pred - y) / np.sum(w)
    # sigmoid output
    s = y_pred
    dz = (dy * s * (1.0 - s))[None, :]
    h_prev = cache[-2]
    gl[-1][0][...] = dz @ h_prev.T
    gl[-1][1][...] = dz.sum(axis=1)
    dh = layers[-1][0].T @ dz
    for li in range(DEPTH - 1, -1, -1):
        z = cache[1 + 2 * li]
        sg = sigmoid(z)
        dsilu = sg * (1.0 + z * (1.0 - sg))
        dz = dh * dsilu
        h_in = cache[2 * li]
        gl[li][0][...] = dz @ h_in.T
        gl[li][1][...] = dz.sum(axis=1)
        dh = layers[li][0].T @ dz
    return loss, grad


class Adam:
    """Adam as published (Kingma and Ba 2014, Algorithm 1): bias-corrected
    first and second moments, update lr m_hat / (sqrt(v_hat) + eps)."""

    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def balance_edges(n_bins: int = 32, lo: float = 1e-8, hi: float = 1.0) -> np.ndarray:
    """n_bins + 1 bin edges equally spaced in log r on [lo, hi], as float32."""
    return (lo * (hi / lo) ** (np.arange(n_bins + 1) / n_bins)).astype(np.float32)


def balance_weights(r: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """Per-sample weights that make every probability range count equally
    (the data balancing of Sec. 3.2).  Sample i falls in bin b = (number of
    edges[1:-1] <= r_i) (values beyond the outer edges go to the outer bins);
    weight n / (count_b * number of non-empty bins), so the weights average
    to 1 and every non-empty bin carries the same total weight."""
    r32 = np.asarray(r, dtype=np.float32)
    inner = np.asarray(edges, dtype=np.float32)[1:-1]
    b = np.searchsorted(inner, r32, side="right")
    n_bins = inner.shape[0] + 1
    cnt = np.bincount(b, minlength=n_bins).astype(np.float64)
    return r32.shape[0] / (cnt[b] * np.count_nonzero(cnt))
