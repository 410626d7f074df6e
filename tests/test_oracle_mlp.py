"""Pins of the FP64 network oracle: finite-difference gradients, closed-form
special cases, Adam against an independent implementation (torch.optim.Adam,
CPU, float64) and the closed form of its first step, and the balancing
weights' defining property."""
import numpy as np
import pytest

from oracle import mlp


def _data(n=64, seed=0):
    rng = np.random.default_rng(seed)
    f = rng.normal(size=(6, n))
    y = rng.uniform(0.05, 0.95, n)
    w = rng.uniform(0.5, 2.0, n)
    return f, y, w


def test_param_count():
    assert mlp.n_params() == 12993


def test_gradient_matches_central_differences():
    theta = mlp.init_params(1)
    f, y, w = _data()
    loss, g = mlp.backward(theta, f, y, w)
    rng = np.random.default_rng(2)
    idx = rng.choice(theta.shape[0], 300, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.mae_loss(mlp.forward(tp, f)[0], y, w) - mlp.mae_loss(mlp.forward(tm, f)[0], y, w)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9


def test_gradient_matches_autograd():
    torch = pytest.importorskip("torch")
    theta = mlp.init_params(3)
    f, y, w = _data(40, 4)
    _, g = mlp.backward(theta, f, y, w)
    t = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    at, h = 0, torch.tensor(f, dtype=torch.float64)
    for li, (o, i) in enumerate(mlp.layer_shapes()):
        W = t[at:at + o * i].reshape(o, i)
        at += o * i
        b = t[at:at + o]
        at += o
        z = W @ h + b[:, None]
        h = torch.sigmoid(z) * z if li < mlp.DEPTH else torch.sigmoid(z)
    yt = torch.tensor(y)
    wt = torch.tensor(w)
    loss = (wt * (h[0] - yt).abs()).sum() / wt.sum()
    loss.backward()
    assert np.allclose(t.grad.numpy(), g, rtol=1e-10, atol=1e-14)


def test_forward_special_cases():
    theta = np.zeros(mlp.n_params())
    f, _, _ = _data(10)
    y, _ = mlp.forward(theta, f)
    assert np.allclose(y, 0.5)  # all-zero network: sigmoid(0)
    # only the output bias set: sigmoid(b4) for any input
    theta[-1] = np.log(3.0)
    y, _ = mlp.forward(theta, f)
    assert np.allclose(y, 0.75)
    # silu at known points
    assert mlp.silu(0.0) == 0.0
    assert mlp.silu(40.0) == pytest.approx(40.0, rel=1e-15)
    assert abs(mlp.silu(-40.0)) < 1e-15


def test_single_path_network_closed_form():
    # one live unit per layer: y = sigmoid(c4 silu(c3 silu(c2 silu(c1 silu(c0 f0)))))
    theta = np.zeros(mlp.n_params())
    L = mlp.unpack(theta)
    cs = [0.7, -1.3, 0.9, 1.1, 2.0]
    L[0][0][0, 0] = cs[0]
    for li in (1, 2, 3):
        L[li][0][0, 0] = cs[li]
    L[4][0][0, 0] = cs[4]
    f = np.zeros((6, 3))
    f[0] = [-1.0, 0.3, 2.5]
    h = f[0]
    for c in cs[:4]:
        z = c * h
        h = z / (1 + np.exp(-z))
    expect = 1 / (1 + np.exp(-cs[4] * h))
    # the other 63 units of each layer see silu(0) = 0 and contribute nothing
    assert np.allclose(mlp.forward(theta, f)[0], expect, rtol=1e-15)


def test_mae_subgradient_zero_at_equality():
    theta = np.zeros(mlp.n_params())
    f = np.zeros((6, 4))
    y = np.full(4, 0.5)  # equals the all-zero network's output
    loss, g = mlp.backward(theta, f, y)
    assert loss == 0.0 and np.all(g == 0.0)


def test_adam_matches_torch_and_first_step_closed_form():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    theta = rng.normal(size=50)
    opt = mlp.Adam(50)
    t = torch.tensor(theta.copy(), requires_grad=True)
    topt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-7)
    th = theta.copy()
    for it in range(5):
        g = rng.normal(size=50)
        new = opt.step(th, g)
        if it == 0:  # m_hat = g, v_hat = g^2
            assert np.allclose(new, th - 1e-3 * g / (np.abs(g) + 1e-7), rtol=1e-14)
        th = new
        t.grad = torch.tensor(g)
        topt.step()
        assert np.allclose(t.detach().numpy(), th, rtol=1e-12, atol=1e-15)


def test_balance_weights_equalise_bins():
    rng = np.random.default_rng(6)
    r = 10 ** (-12 * rng.uniform(0, 1, 100000) ** 2)  # skewed toward large r
    edges = mlp.balance_edges(12, 1e-12, 1.0)
    assert np.allclose(np.log10(edges.astype(np.float64)), np.linspace(-12, 0, 13), atol=1e-6)
    w = mlp.balance_weights(r, edges)
    # brute force: the bin of each sample by scanning the edges
    b = np.array([sum(1 for e in edges[1:-1] if e <= np.float32(x)) for x in r[:2000]])
    assert np.array_equal(b, np.searchsorted(edges[1:-1], r[:2000].astype(np.float32), side="right"))
    full_b = np.searchsorted(edges[1:-1], r.astype(np.float32), side="right")
    per_bin = np.bincount(full_b, weights=w, minlength=12)
    nz = per_bin[per_bin > 0]
    assert np.allclose(nz, nz[0])
    assert w.mean() == pytest.approx(1.0)


def test_features_sign_and_scale():
    u = np.array([[0.0, 1.0, -1.0]], dtype=np.float64).repeat(3, 0)
    k = np.array([[1e-4, -1e-4, 0.0]]).repeat(3, 0)
    f = mlp.features(u, k)
    assert np.allclose(f[0], [0.0, np.log(2) / 7, -np.log(2) / 7])
    assert np.allclose(f[3], [np.log(2) / 10, -np.log(2) / 10, 0.0])


def test_invariant_features_match_the_pinned_invariants():
    # x and v of the numpy features against the C oracle's invariants (pinned
    # at 50 digits in test_oracle_physics), including collinear gamma = 1e3
    import oracle
    from paper_2206_02937_gb300 import workloads as wl
    rng = np.random.default_rng(12)
    u, k = wl.c3(500, seed=8)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    u[:, :20] = (np.sqrt(1e6 - 1.0) * d)[:, None]
    k[:, :20] = np.logspace(-4, 0, 20)[None, :] * (d[:, None] + 1e-4 * rng.normal(size=(3, 20)))
    x, v = mlp.pair_invariants(u, k)
    for i in range(500):
        xr, vr = oracle.invariants(u[:, i], k[:, i])
        assert abs(x[i] / xr - 1) < 1e-8 and abs(v[i] / vr - 1) < 1e-8, i
    f = mlp.features(u, k, mode="invariants")
    assert np.allclose(f[0], np.log(x) / 8) and np.allclose(f[1], np.log(v) / 8)
    assert not f[2:].any()
