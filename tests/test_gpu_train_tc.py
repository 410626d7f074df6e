"""Training of the surrogate network with every contraction on the tcgen05
tensor cores (compton_mlp_set_train_precision(MODE_MLP_BF16)), against the
FP64 oracle (Sec. 3.2: MAE loss, Adam).

  * gradients: per tensor, relative Frobenius error <= 2e-2 (BF16 operands,
    FP32 accumulation), on ragged batches (not a multiple of the 128-row tile),
    with sample weights, in both input modes, and on batches of more tiles than
    there are SMs (several tiles per CTA, the weight gradients accumulated in
    tensor memory across them);
  * the loss within 1e-2 relative; Adam on the GPU's own gradient as the
    oracle's Adam;
  * learning: on samples of the analytic target the loss falls, and the
    trained network's error is a fraction of the untrained one's.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

BF16_GRAD_TOL = 2e-2


def _run_step(cg, torch, n, weighted, feat, seed):
    """One BF16 training step and the oracle's gradient on the same batch.
    The MAE subgradient w sign(y' - y) jumps where the prediction meets the
    target, so a sample within BF16 rounding of its target could take the
    other sign than in FP64; the targets are therefore drawn at least 0.05
    away from the oracle's own prediction, on either side."""
    u, k = wl.c3(n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    w = rng.uniform(0.5, 2.0, n) if weighted else None
    th = omlp.init_params(seed + 2).astype(np.float32)
    f = omlp.features(u, k, mode="invariants" if feat else "momenta")
    y_pred = omlp.forward(th.astype(np.float64), f)
    y_pred = y_pred[0] if isinstance(y_pred, tuple) else y_pred
    side = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    y = np.clip(np.ravel(y_pred) + side * rng.uniform(0.05, 0.3, n), 0.0, 1.0)
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1, max_train_batch=n)
    try:
        cg.compton_mlp_set_params(ctx, th)
        cg.compton_mlp_set_features(ctx, feat)
        cg.compton_mlp_set_train_precision(ctx, cg.MODE_MLP_BF16)
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        yt = torch.from_numpy(y.astype(np.float32)).cuda()
        wt = None if w is None else torch.from_numpy(w.astype(np.float32)).cuda()
        loss = cg.compton_mlp_train_step(ctx, ut, kt, yt, wt, lr=1e-3)
        assert cg.compton_check(ctx) == cg.COMPTON_OK
        g_gpu = cg.compton_mlp_get_grad(ctx).astype(np.float64)
        th_new = cg.compton_mlp_get_params(ctx).astype(np.float64)
    finally:
        cg.compton_destroy(ctx)
    loss_ref, g_ref = omlp.backward(th.astype(np.float64), f, y, w)
    return th, loss, loss_ref, g_gpu, g_ref, th_new


@pytest.mark.parametrize("n,weighted,feat", [(1000, False, 0), (4097, True, 0), (2500, False, 1),
                                             (40001, True, 0)])
def test_tensor_core_gradient_matches_oracle(n, weighted, feat):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    th, loss, loss_ref, g_gpu, g_ref, th_new = _run_step(cg, torch, n, weighted, feat, 31 + n)
    assert loss == pytest.approx(loss_ref, rel=1e-2)
    G_gpu, G_ref = omlp.unpack(g_gpu), omlp.unpack(g_ref)
    errs = []
    for (Wg, bg), (Wr, br) in zip(G_gpu, G_ref):
        errs.append((np.linalg.norm(Wg - Wr) / np.linalg.norm(Wr), np.linalg.norm(bg - br) / np.linalg.norm(br)))
    print(f"\nn={n} weighted={weighted} feat={feat}: relative Frobenius errors per layer (W, b): "
          + ", ".join(f"({a:.1e}, {b:.1e})" for a, b in errs))
    for ew, eb in errs:
        assert ew <= BF16_GRAD_TOL and eb <= BF16_GRAD_TOL
    opt = omlp.Adam(th.shape[0])
    th_ref = opt.step(th.astype(np.float64), g_gpu)
    assert np.allclose(th_new, th_ref, rtol=1e-5, atol=1e-7)


def test_tensor_core_gradient_equals_fp32_path_closely():
    """Both training precisions on the same batch: the BF16 tensor-core
    gradient is within the BF16 bound of the FP32 CUDA-core one."""
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    n = 3000
    u, k = wl.c3(n, seed=71)
    y = np.random.default_rng(72).uniform(0.02, 0.98, n).astype(np.float32)
    th = omlp.init_params(73).astype(np.float32)
    grads = []
    for prec in (cg.MODE_MLP_FP32, cg.MODE_MLP_BF16):
        ctx = cg.compton_init(1, 0, 1.0, 0.05, 1, max_train_batch=n)
        try:
            cg.compton_mlp_set_params(ctx, th)
            cg.compton_mlp_set_train_precision(ctx, prec)
            cg.compton_mlp_train_step(ctx, torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda(),
                                      torch.from_numpy(y).cuda(), None, lr=0.0)
            grads.append(omlp.unpack(cg.compton_mlp_get_grad(ctx).astype(np.float64)))
        finally:
            cg.compton_destroy(ctx)
    for (W32, b32), (W16, b16) in zip(*grads):
        assert np.linalg.norm(W16 - W32) <= BF16_GRAD_TOL * np.linalg.norm(W32)
        assert np.linalg.norm(b16 - b32) <= BF16_GRAD_TOL * np.linalg.norm(b32)


def test_tensor_core_training_reduces_error():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    n_train, n_test, batch = 65536, 8192, 4096
    u, k = wl.c3(n_train + n_test, seed=41)
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1, max_train_batch=batch)
    try:
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        r = torch.zeros(n_train + n_test, device="cuda")
        cg.compton_kn_ratio(ctx, ut, kt, r)
        cg.compton_mlp_set_params(ctx, omlp.init_params(5).astype(np.float32))
        cg.compton_mlp_set_train_precision(ctx, cg.MODE_MLP_BF16)
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
        assert cg.compton_check(ctx) == cg.COMPTON_OK
    finally:
        cg.compton_destroy(ctx)
    ls = [l_ for l_ in losses if l_ is not None]
    assert ls[-1] < 0.5 * ls[0]
    assert mae1 < 0.5 * mae0, (mae0, mae1)


def test_train_precision_rejects_other_modes():
    import paper_2206_02937_gb300 as cg
    torch_cuda()
    cg.build()
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1, max_train_batch=16)
    try:
        for bad in (cg.MODE_PLAIN, cg.MODE_MLP_FP8, 99):
            with pytest.raises(cg.ComptonError) as e:
                cg.compton_mlp_set_train_precision(ctx, bad)
            assert e.value.status == cg.COMPTON_EINVAL
    finally:
        cg.compton_destroy(ctx)
