"""Parity of the surrogate network's GPU forward (FP32 CUDA cores; BF16 and FP8
E4M3 tensor cores) with the FP64 oracle forward on the same parameters and
inputs, and the save/load round trip.

Tolerances (derived from the operand precisions; the output is a sigmoid in
[0, 1]):
  * FP32: |dr| <= 2e-6 (64-term FP32 dot products, exact exp);
  * BF16: |dr| <= 2e-2, mean <= 4e-3 (8-bit mantissas on every operand of four
    layers, hardware tanh in SiLU);
  * FP8 E4M3: |dr| <= 0.12, mean <= 0.03 (4-bit mantissas, per-tensor scales).
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _theta(seed, gain=1.0):
    th = omlp.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for W, b in omlp.unpack(th):
        W *= gain
        b[...] = rng.normal(0, 0.1, b.shape)
    return th


def _run(torch, theta, u, k, modes, calibrate=True, features=0):
    import paper_2206_02937_gb300 as cg
    cg.build()
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1)
    try:
        cg.compton_mlp_set_params(ctx, theta.astype(np.float32))
        cg.compton_mlp_set_features(ctx, features)
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        if calibrate:
            cg.compton_mlp_calibrate(ctx, ut, kt)
        out = {}
        for mode in modes:
            r = torch.full((u.shape[1],), -1.0, device="cuda")
            cg.compton_mlp_infer(ctx, ut, kt, mode, r)
            torch.cuda.synchronize()
            out[mode] = r.cpu().numpy().astype(np.float64)
        assert cg.compton_check(ctx) == cg.COMPTON_OK
        blob = cg.compton_mlp_save(ctx)
    finally:
        cg.compton_destroy(ctx)
    return out, blob


@pytest.mark.parametrize("n", [1, 127, 128, 129, 5000, 70001])
def test_forward_parity_all_modes(n):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    u, k = wl.c3(n, seed=20 + n % 7)
    th = _theta(1, gain=1.5)
    ref, _ = omlp.forward(th.astype(np.float32).astype(np.float64), omlp.features(u, k))
    out, _ = _run(torch, th, u, k, [cg.MODE_MLP_FP32, cg.MODE_MLP_BF16, cg.MODE_MLP_FP8])
    e32 = np.abs(out[cg.MODE_MLP_FP32] - ref)
    assert e32.max() <= 2e-6, e32.max()
    e16 = np.abs(out[cg.MODE_MLP_BF16] - ref)
    assert e16.max() <= 2e-2 and e16.mean() <= 4e-3, (e16.max(), e16.mean())
    e8 = np.abs(out[cg.MODE_MLP_FP8] - ref)
    assert e8.max() <= 0.12 and e8.mean() <= 0.03, (e8.max(), e8.mean())


def test_tensor_core_layout_with_structured_weights():
    # weights exactly representable in BF16 and a single live path through
    # each layer: any transposition or swizzle error moves the output far
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    th = np.zeros(omlp.n_params())
    L = omlp.unpack(th)
    L[0][0][5, 2] = 1.0          # unit 5 of layer 1 reads feature 2 (u_z)
    L[1][0][17, 5] = 2.0         # unit 17 of layer 2 reads unit 5
    L[2][0][40, 17] = 0.5
    L[3][0][63, 40] = 1.25
    L[4][0][0, 63] = 3.0
    u, k = wl.c3(1000, seed=3)
    ref, _ = omlp.forward(th, omlp.features(u, k))
    out, _ = _run(torch, th, u, k, [cg.MODE_MLP_BF16, cg.MODE_MLP_FP32])
    assert np.abs(out[cg.MODE_MLP_FP32] - ref).max() <= 2e-6
    assert np.abs(out[cg.MODE_MLP_BF16] - ref).max() <= 1e-2
    assert np.std(ref) > 0.02  # the path actually varies with the input


def test_save_load_round_trip_bit_exact():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    u, k = wl.c3(3000, seed=5)
    th = _theta(2)
    out, blob = _run(torch, th, u, k, [cg.MODE_MLP_BF16, cg.MODE_MLP_FP8])
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1)
    try:
        cg.compton_mlp_load(ctx, blob)
        assert np.array_equal(cg.compton_mlp_get_params(ctx), th.astype(np.float32))
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        for mode in (cg.MODE_MLP_BF16, cg.MODE_MLP_FP8):
            r = torch.zeros(3000, device="cuda")
            cg.compton_mlp_infer(ctx, ut, kt, mode, r)
            torch.cuda.synchronize()
            assert np.array_equal(r.cpu().numpy().astype(np.float64), out[mode])
        bad = bytearray(blob)
        bad[0:4] = b"XXXX"
        with pytest.raises(cg.ComptonError):
            cg.compton_mlp_load(ctx, bytes(bad))
    finally:
        cg.compton_destroy(ctx)


@pytest.mark.parametrize("n", [129, 5000])
def test_forward_parity_invariant_features(n):
    # inputs ln(x)/8, ln(v)/8 from the FP32 invariants (relative error ~1e-6)
    # against the FP64 oracle's: FP32 bound 5e-6, the others as above
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    u, k = wl.c3(n, seed=40 + n % 5)
    th = _theta(3, gain=1.5)
    ref, _ = omlp.forward(th.astype(np.float32).astype(np.float64), omlp.features(u, k, mode="invariants"))
    out, blob = _run(torch, th, u, k, [cg.MODE_MLP_FP32, cg.MODE_MLP_BF16, cg.MODE_MLP_FP8],
                     features=cg.FEATURES_INVARIANTS)
    e32 = np.abs(out[cg.MODE_MLP_FP32] - ref)
    assert e32.max() <= 5e-6, e32.max()
    e16 = np.abs(out[cg.MODE_MLP_BF16] - ref)
    assert e16.max() <= 2e-2 and e16.mean() <= 4e-3, (e16.max(), e16.mean())
    e8 = np.abs(out[cg.MODE_MLP_FP8] - ref)
    assert e8.max() <= 0.12 and e8.mean() <= 0.03, (e8.max(), e8.mean())
    # the mode travels with a saved network
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1)
    try:
        cg.compton_mlp_load(ctx, blob)
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        r = torch.zeros(n, device="cuda")
        cg.compton_mlp_infer(ctx, ut, kt, cg.MODE_MLP_FP32, r)
        torch.cuda.synchronize()
        assert np.array_equal(r.cpu().numpy().astype(np.float64), out[cg.MODE_MLP_FP32])
        with pytest.raises(cg.ComptonError):
            cg.compton_mlp_set_features(ctx, 7)
    finally:
        cg.compton_destroy(ctx)


def test_no_model_is_reported():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1)
    try:
        u = torch.zeros((3, 10), device="cuda")
        r = torch.zeros(10, device="cuda")
        with pytest.raises(cg.ComptonError) as e:
            cg.compton_mlp_infer(ctx, u, u, cg.MODE_MLP_BF16, r)
        assert e.value.status == cg.COMPTON_ENOMODEL
    finally:
        cg.compton_destroy(ctx)
