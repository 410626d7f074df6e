"""The GPU's scattering-angle sampler against the oracle's inverse CDF, draw by
draw (including the 24-bit tails near forward and backward scattering), and
the distribution of GPU samples against the analytic Klein-Nishina angular
distribution (chi-square)."""
import math

import numpy as np
import pytest

import oracle
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

XS = [1e-6, 1e-4, 1e-2, 0.3, 1.0, 7.0, 100.0, 3000.0]


def _run(torch, x, r):
    import paper_2206_02937_gb300 as cg
    cg.build()
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1)
    try:
        xt = torch.from_numpy(np.asarray(x, dtype=np.float32)).cuda()
        rt = torch.from_numpy(np.asarray(r, dtype=np.uint32).view(np.int32)).cuda()
        c = torch.empty_like(xt)
        s = torch.empty_like(xt)
        q = torch.empty_like(xt)
        cg.compton_kn_sample_angle(ctx, xt, rt, c, s, q)
        torch.cuda.synchronize()
        return c.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64), q.cpu().numpy()
    finally:
        cg.compton_destroy(ctx)


def test_draw_by_draw_including_tails():
    torch = torch_cuda()
    r24 = np.array([0, 1, 2, 100, 2**22, 2**23 - 1, 2**23, 2**23 + 1, 2**24 - 101, 2**24 - 3, 2**24 - 2, 2**24 - 1]
                   + list(np.random.default_rng(0).integers(0, 2**24, 200)), dtype=np.int64)
    xs, rs = [], []
    for x in XS:
        xs += [x] * len(r24)
        rs += list((r24 << 8) | 0x5A)
    cth, sth, ratio = _run(torch, xs, rs)
    for i, (x, r) in enumerate(zip(xs, rs)):
        x32 = float(np.float32(x))
        u1 = ((r >> 8) + 0.5) / 2**24
        t = oracle.kn_sample_t(x32, u1)
        c_ref, s_ref = 1.0 - t, math.sqrt(t * (2.0 - t))
        # angle error in radians, and the Compton ratio
        assert math.hypot(cth[i] - c_ref, sth[i] - s_ref) < 3e-6, (x, r >> 8, cth[i], c_ref, sth[i], s_ref)
        # d ratio / ratio = x ratio dt: at x = 3e3 an FP32 t gives a few 1e-6
        assert ratio[i] == pytest.approx(1.0 / (1.0 + x32 * t), rel=1e-5)


@pytest.mark.parametrize("x", [1e-4, 1e-2, 1.0, 100.0])
def test_gpu_angle_distribution_chi_square(x):
    from scipy.stats import chi2
    torch = torch_cuda()
    n = 1_000_000
    r = np.random.default_rng(int(x * 1000) + 1).integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    cth, _, _ = _run(torch, np.full(n, x), r)
    x32 = float(np.float32(x))
    t = 1.0 - cth
    edges = np.linspace(0.0, 2.0, 51)
    counts, _ = np.histogram(np.clip(t, 0, 2), edges)
    tot = oracle.kn_cdf(x32, 2.0)
    probs = np.array([oracle.kn_cdf(x32, b) - oracle.kn_cdf(x32, a) for a, b in zip(edges[:-1], edges[1:])]) / tot
    exp = probs * n
    stat = float(((counts - exp) ** 2 / exp).sum())
    assert chi2.sf(stat, 49) > 1e-3
