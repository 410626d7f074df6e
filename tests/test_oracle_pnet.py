"""Pins of the FP64 oracle of the paper's 9-12-9 network: parameter count,
central-difference gradients, a single live path with a closed form, ReLU and
sigmoid special cases, and the feature map."""
import numpy as np

from oracle import pnet
from paper_2206_02937_gb300 import workloads as wl


def test_param_count():
    assert pnet.N_PARAMS == 9 * 9 + 9 + 12 * 9 + 12 + 9 * 12 + 9 + 9 + 1 == 337


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    th = pnet.init_params(1)
    for W, b in pnet.unpack(th):
        b[...] = rng.normal(0, 0.3, b.shape)
    f = rng.normal(0, 1.0, (9, 40))
    y = rng.uniform(0.05, 0.95, 40)
    w = rng.uniform(0.5, 2.0, 40)
    _, g = pnet.backward(th, f, y, w)
    h = 1e-6
    for i in rng.choice(pnet.N_PARAMS, 60, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (pnet.backward(tp, f, y, w)[0] - pnet.backward(tm, f, y, w)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(g[i]), (i, fd, g[i])


def test_single_path_closed_form():
    th = np.zeros(pnet.N_PARAMS)
    L = pnet.unpack(th)
    L[0][0][2, 4] = 1.5      # unit 2 reads feature 4
    L[1][0][7, 2] = 2.0
    L[2][0][3, 7] = 0.5
    L[3][0][0, 3] = 1.2
    L[3][1][0] = -0.3
    f = np.zeros((9, 3))
    f[4] = [-1.0, 0.25, 2.0]
    y, _ = pnet.forward(th, f)
    z = 1.2 * 0.5 * 2.0 * np.maximum(1.5 * f[4], 0.0) - 0.3
    assert np.allclose(y, 1.0 / (1.0 + np.exp(-z)), rtol=1e-15)
    assert y[0] == 1.0 / (1.0 + np.exp(0.3))  # negative input: the ReLU stops the path


def test_features():
    u, k = wl.c3(100, seed=4)
    f = pnet.features(u, k, 1.0 / 64, 1.0 / 64, 0.1)
    assert f.shape == (9, 100)
    assert np.allclose(f[0], np.sign(u[0]) * np.log1p(np.abs(u[0])) / 7.0)
    assert np.allclose(f[6:8], np.log(1.0 / 64) / 8.0) and np.allclose(f[8], np.log(0.1) / 8.0)
