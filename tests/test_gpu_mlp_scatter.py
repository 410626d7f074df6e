"""The surrogate modes of compton_scatter_step: in-range pairs take
P = 1 - exp(-2 n dt r) with r from the network (the GPU's own inference on
the same pair), out-of-range pairs fall back to the analytic probability, and
every collision matches the oracle's collision with the pair's own draws."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import _dev_array, energy_scale, species_np, to_species, torch_cuda

pytestmark = pytest.mark.gpu


def _workload(seed=3):
    w = wl.c2(48, 48, 40, seed=seed)
    rng = wl.rng_for(seed + 50)
    # push some pairs outside the network's range: gamma > 1e3, eps < 1e-4, eps > 1
    ne, ng = w.n_e, w.n_g
    for frac, scale, sp in ((0.02, 3e3, w.e), (0.02, 3e-5 / 1e-2, w.g), (0.01, 300.0, w.g)):
        idx = rng.choice(sp["ux"].shape[0], int(frac * sp["ux"].shape[0]), replace=False)
        for c in ("ux", "uy", "uz"):
            sp[c][idx] = (sp[c][idx] * scale).astype(np.float32)
    _ = (ne, ng)
    return w


@pytest.mark.parametrize("mode_name", ["MODE_MLP_BF16", "MODE_MLP_FP32"])
def test_surrogate_scatter_matches_network_and_oracle(mode_name):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    mode = getattr(cg, mode_name)
    w = _workload()
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        cg.compton_mlp_set_params(ctx, omlp.init_params(9).astype(np.float32))
        e_in, g_in = to_species(torch, w.e), to_species(torch, w.g)
        e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
        pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 0)
        torch.cuda.synchronize()
        be, bg = species_np(e_out), species_np(g_out)
        off_e = _dev_array(torch, pairs.off_e_dev, w.n_cells + 1).astype(np.int64)
        off_g = _dev_array(torch, pairs.off_g_dev, w.n_cells + 1).astype(np.int64)
        m = np.minimum(np.diff(off_e), np.diff(off_g))
        cell = np.repeat(np.arange(w.n_cells), m)
        j = np.arange(cell.shape[0]) - np.concatenate([[0], np.cumsum(m)])[cell]
        ie, ig = off_e[cell] + j, off_g[cell] + j
        n = cell.shape[0]
        # the network's r on the same pairs, through the inference entry point
        u = np.stack([be[c][ie] for c in ("ux", "uy", "uz")]).astype(np.float32)
        k = np.stack([bg[c][ig] for c in ("ux", "uy", "uz")]).astype(np.float32)
        r = torch.zeros(n, device="cuda")
        cg.compton_mlp_infer(ctx, torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda(), mode, r)
        P = torch.zeros(n, device="cuda")
        F = torch.zeros(n, dtype=torch.uint8, device="cuda")
        cg.compton_get_stats(ctx, reset=True)
        cg.compton_scatter_step(ctx, e_out, g_out, pairs, mode, 0, P, F)
        st = cg.compton_get_stats(ctx, reset=True)
        ae, ag = species_np(e_out), species_np(g_out)
        r, P, F = r.cpu().numpy().astype(np.float64), P.cpu().numpy().astype(np.float64), F.cpu().numpy()
    finally:
        cg.compton_destroy(ctx)
    dens = np.maximum(np.diff(off_e), np.diff(off_g))[cell] * w.w_over_v
    g2 = 1.0 + (u.astype(np.float64) ** 2).sum(0)
    e2 = (k.astype(np.float64) ** 2).sum(0)
    in_range = (g2 <= 1e6) & (e2 >= 1e-8) & (e2 <= 1.0)
    assert st["mlp_fallbacks"] == int((~in_range).sum()) > 0
    P_net = 1.0 - np.exp(-2.0 * dens * w.dt * r)
    assert np.allclose(P[in_range], P_net[in_range], rtol=1e-5, atol=1e-9)
    P_ana = np.array([oracle.scatter_event(u[:, q], k[:, q], dens[q], w.dt, w.seed, 0, q)[2]
                      for q in np.nonzero(~in_range)[0]])
    assert np.allclose(P[~in_range], P_ana, rtol=2e-5, atol=1e-9)
    u0 = np.array([oracle.bernoulli_u0(w.seed, 0, q) for q in range(n)])
    ref_flag = (u0 < P).astype(np.uint8)
    assert np.array_equal(F, ref_flag)
    hit = np.nonzero(F)[0]
    assert hit.size > 50
    scale = energy_scale(u, k)
    for q in hit[:400]:
        uo, ko = oracle.collide(u[:, q].astype(np.float64), k[:, q].astype(np.float64), w.seed, 0, int(q))
        ua = np.array([ae[c][ie[q]] for c in ("ux", "uy", "uz")], dtype=np.float64)
        ka = np.array([ag[c][ig[q]] for c in ("ux", "uy", "uz")], dtype=np.float64)
        assert np.linalg.norm(ua - uo) <= 1e-5 * scale[q]
        assert np.linalg.norm(ka - ko) <= 1e-5 * scale[q]


@pytest.mark.parametrize("mode_name", ["MODE_MLP_BF16", "MODE_MLP_FP32", "MODE_PNET"])
def test_surrogate_filtered_equals_full_evaluation(mode_name):
    # the surrogate step without prob_out runs the network on the candidates
    # of the probability kernel's filter only; flags and momenta equal those
    # of the full evaluation (every pair a candidate)
    import paper_2206_02937_gb300 as cg
    from oracle import pnet as opn
    torch = torch_cuda()
    cg.build()
    mode = getattr(cg, mode_name)
    w = _workload(seed=4)
    out = {}
    for want_p in (True, False):
        ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
        try:
            cg.compton_mlp_set_params(ctx, omlp.init_params(11).astype(np.float32))
            cg.compton_pnet_set_params(ctx, opn.init_params(12).astype(np.float32))
            e_in, g_in = to_species(torch, w.e), to_species(torch, w.g)
            e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
            pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 2)
            n = pairs.max_pairs
            P = torch.zeros(n, device="cuda") if want_p else None
            F = torch.zeros(n, dtype=torch.uint8, device="cuda")
            cg.compton_get_stats(ctx, reset=True)
            cg.compton_scatter_step(ctx, e_out, g_out, pairs, mode, 2, P, F)
            st = cg.compton_get_stats(ctx, reset=True)
            out[want_p] = (F.cpu().numpy(), species_np(e_out), species_np(g_out), st)
        finally:
            cg.compton_destroy(ctx)
    (Fa, ea, ga, sa), (Fb, eb, gb, sb) = out[True], out[False]
    assert np.array_equal(Fa, Fb) and Fa.sum() > 20
    assert sa["scatters"] == sb["scatters"] and sa["pairs_tested"] == sb["pairs_tested"]
    assert sb["mlp_fallbacks"] <= sa["mlp_fallbacks"]  # only candidates are looked at
    for c in ("ux", "uy", "uz"):
        assert np.array_equal(ea[c], eb[c]) and np.array_equal(ga[c], gb[c])
