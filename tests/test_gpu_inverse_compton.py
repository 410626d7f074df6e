"""The inverse-Compton benchmark of Sec. 3.3 on the analytic path: an
electron beam (p_e along +x) through an isotropic photon gas at eps = 2.5.
Deep in the Klein-Nishina regime the photon takes most of the electron's
energy, so the spectrum of scattered photons peaks near p_e (the paper
reports the peak at p_gamma ~ p_e).  A photon scattered twice can end above
gamma + eps, so the bound checked is the conservation of the totals: equal
weights make the sum of gamma plus the sum of |k| (and the summed momentum)
invariant up to FP32 rounding."""
import numpy as np
import pytest

from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p_e", [25.0, 100.0])
def test_spectrum_peaks_near_beam_momentum(p_e):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w = wl.inverse_compton(p_e, n_cells=64, ppc=64)
    ctx = cg.compton_init(w.n_cells, w.n_e, w.w_over_v, w.dt, w.seed)
    try:
        def sp(d):
            return cg.Species(*(torch.from_numpy(d[c] if c != "id" else d[c].view(np.int32)).cuda()
                                for c in ("ux", "uy", "uz", "cell", "id")))
        bufs = [[sp(w.e), sp(w.g)], None]
        bufs[1] = [cg.Species.empty_like(bufs[0][0]), cg.Species.empty_like(bufs[0][1])]
        steps = 400 if p_e < 50 else 1200
        for i in range(steps):
            src, dst = bufs[i % 2], bufs[(i + 1) % 2]
            pr = cg.compton_bin_pairs(ctx, src[0], src[1], dst[0], dst[1], i)
            cg.compton_scatter_step(ctx, dst[0], dst[1], pr, cg.MODE_PLAIN, i)
        torch.cuda.synchronize()
        out = bufs[steps % 2][1]
        k = torch.stack([out.ux, out.uy, out.uz]).double().cpu().numpy()
        oe = bufs[steps % 2][0]
        u = torch.stack([oe.ux, oe.uy, oe.uz]).double().cpu().numpy()
    finally:
        cg.compton_destroy(ctx)
    eps = np.linalg.norm(k, axis=0)
    hit = np.abs(eps - 2.5) > 1e-4
    assert hit.sum() > 0.1 * eps.size
    u0 = np.stack([w.e["ux"], w.e["uy"], w.e["uz"]]).astype(np.float64)
    k0 = np.stack([w.g["ux"], w.g["uy"], w.g["uz"]]).astype(np.float64)
    e_tot0 = np.sqrt(1.0 + (u0 * u0).sum(0)).sum() + np.linalg.norm(k0, axis=0).sum()
    e_tot = np.sqrt(1.0 + (u * u).sum(0)).sum() + eps.sum()
    assert abs(e_tot - e_tot0) <= 1e-5 * e_tot0
    p_tot0, p_tot = (u0 + k0).sum(1), (u + k).sum(1)
    assert np.all(np.abs(p_tot - p_tot0) <= 1e-5 * e_tot0)
    h, edges = np.histogram(np.log10(eps[hit]), bins=70, range=(-1.0, 2.5))
    peak = 10 ** (0.5 * (edges[np.argmax(h)] + edges[np.argmax(h) + 1]))
    assert 0.6 * p_e <= peak <= 1.1 * p_e, peak
