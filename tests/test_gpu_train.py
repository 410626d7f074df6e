"""Training of the surrogate network on the GPU by the library's own forward,
backward and Adam kernels, against the FP64 oracle.

  * gradients: per tensor, relative Frobenius error <= 1e-4 (FP32 kernels);
  * Adam: the GPU update equals the oracle's Adam applied to the GPU gradient;
  * learning: on samples of the analytic target the loss falls, and the
    trained network's error is a fraction of the untrained one's.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _ctx(cg, batch):
    return cg.compton_init(1, 0, 1.0, 0.05, 1, max_train_batch=batch)


def _tensors(torch, u, k, y, w):
    return (torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda(), torch.from_numpy(y.astype(np.float32)).cuda(),
            None if w is None else torch.from_numpy(w.astype(np.float32)).cuda())


@pytest.mark.parametrize("n,weighted,feat", [(1000, False, 0), (4097, True, 0), (2500, False, 1)])
def test_gradient_and_adam_match_oracle(n, weighted, feat):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    u, k = wl.c3(n, seed=31)
    rng = np.random.default_rng(32)
    y = rng.uniform(0.02, 0.98, n)
    w = rng.uniform(0.5, 2.0, n) if weighted else None
    th = omlp.init_params(7).astype(np.float32)
    ctx = _ctx(cg, n)
    try:
        cg.compton_mlp_set_params(ctx, th)
        cg.compton_mlp_set_features(ctx, feat)
        ut, kt, yt, wt = _tensors(torch, u, k, y, w)
        loss = cg.compton_mlp_train_step(ctx, ut, kt, yt, wt, lr=1e-3)
        g_gpu = cg.compton_mlp_get_grad(ctx).astype(np.float64)
        th_new = cg.compton_mlp_get_params(ctx).astype(np.float64)
    finally:
        cg.compton_destroy(ctx)
    f = omlp.features(u, k, mode="invariants" if feat else "momenta")
    loss_ref, g_ref = omlp.backward(th.astype(np.float64), f, y, w)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    G_gpu, G_ref = omlp.unpack(g_gpu), omlp.unpack(g_ref)
    for (Wg, bg), (Wr, br) in zip(G_gpu, G_ref):
        assert np.linalg.norm(Wg - Wr) <= 1e-4 * np.linalg.norm(Wr) + 1e-9
        assert np.linalg.norm(bg - br) <= 1e-4 * np.linalg.norm(br) + 1e-9
    # Adam step on the GPU's own gradient (FP32 arithmetic: relative 1e-6)
    opt = omlp.Adam(th.shape[0])
    th_ref = opt.step(th.astype(np.float64), g_gpu)
    assert np.allclose(th_new, th_ref, rtol=1e-5, atol=1e-7)


def test_training_reduces_error_on_analytic_targets():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    n_train, n_test, batch = 65536, 8192, 4096
    u, k = wl.c3(n_train + n_test, seed=41)
    ctx = _ctx(cg, batch)
    try:
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        r = torch.zeros(n_train + n_test, device="cuda")
        cg.compton_kn_ratio(ctx, ut, kt, r)
        cg.compton_mlp_set_params(ctx, omlp.init_params(5).astype(np.float32))
        te = slice(n_train, None)
        r_hat = torch.zeros(n_test, device="cuda")

        def test_mae():
            cg.compton_mlp_infer(ctx, ut[:, te], kt[:, te], cg.MODE_MLP_FP32, r_hat)
            torch.cuda.synchronize()
            return float((r_hat - r[te]).abs().mean())

        mae0 = test_mae()
        losses = []
        gen = torch.Generator(device="cuda").manual_seed(0)
        for it in range(400):
            idx = torch.randint(0, n_train, (batch,), device="cuda", generator=gen)
            ub, kb = ut[:, idx].contiguous(), kt[:, idx].contiguous()
            losses.append(cg.compton_mlp_train_step(ctx, ub, kb, r[idx].contiguous(), None, lr=1e-3,
                                                    want_loss=(it % 20 == 0)))
        mae1 = test_mae()
    finally:
        cg.compton_destroy(ctx)
    ls = [l_ for l_ in losses if l_ is not None]
    assert ls[-1] < 0.5 * ls[0]
    assert mae1 < 0.5 * mae0, (mae0, mae1)


def test_balance_weights_match_oracle():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    u, k = wl.c3(200000, seed=61)
    ctx = _ctx(cg, 16)
    try:
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        r = torch.zeros(200000, device="cuda")
        cg.compton_kn_ratio(ctx, ut, kt, r)
        edges = omlp.balance_edges(32, 1e-8, 1.0)
        w = torch.zeros(200000, device="cuda")
        cg.compton_mlp_balance_weights(ctx, r, edges, w)
        torch.cuda.synchronize()
        rn = r.cpu().numpy()
        ref = omlp.balance_weights(rn, edges)
        assert np.allclose(w.cpu().numpy(), ref, rtol=1e-6)
    finally:
        cg.compton_destroy(ctx)
