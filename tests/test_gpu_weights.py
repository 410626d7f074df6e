"""Unequal macro-particle weights on the GPU against the oracle's weighted
step (pair density max(N_e, N_g) max(w_e, w_g), the per-pair P_max of
Sec. 3.2; weight rejection of the heavier partner):

  * binning carries the weights with the particles: bit-exact;
  * probabilities within FP32 rounding, decisions bit-exact outside the
    1e-6 band around P, which partner takes its new momentum bit-exact (the
    rejection test u w_heavy < w_light is exact on both sides);
  * momenta within 1e-5 (gamma + eps) of the pair; a rejected partner keeps
    its momentum bit for bit;
  * the paper's network in the weighted step sees the pair's own weights
    and P_max;
  * argument checks: weighted input without weighted output, a pair list
    binned with weights used without them, No-Time-Counter with weights.
"""
import numpy as np
import pytest

import oracle
from oracle import pnet as opn
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import _dev_array, energy_scale, species_np, to_species, torch_cuda, u0_of_pairs

pytestmark = pytest.mark.gpu

FLIP_BAND = 1e-6
MOM_TOL = 1e-5


def _weighted(seed, both=True, nx=48, ppc=40):
    w = wl.c2(nx, nx, ppc, seed=seed)
    rng = wl.rng_for(seed + 70)
    e = dict(w.e, w=(w.w_over_v * 10.0 ** rng.uniform(-1.0, 1.0, w.n_e)).astype(np.float32))
    g = dict(w.g, w=(w.w_over_v * 10.0 ** rng.uniform(-1.0, 1.0, w.n_g)).astype(np.float32)) if both else w.g
    return w, e, g


def _mom(s):
    return np.stack([s["ux"], s["uy"], s["uz"]]).astype(np.float64)


def _run(cg, torch, w, e, g, step, mode=None, th=None, want_p=True):
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        if th is not None:
            cg.compton_pnet_set_params(ctx, th)
        e_in, g_in = to_species(torch, e), to_species(torch, g)
        e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
        pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, step)
        torch.cuda.synchronize()
        be, bg = species_np(e_out), species_np(g_out)
        n = max(1, pairs.max_pairs)
        P = torch.zeros(n, device="cuda")
        F = torch.zeros(n, dtype=torch.uint8, device="cuda")
        if not want_p:
            P = None
        cg.compton_get_stats(ctx, reset=True)
        cg.compton_scatter_step(ctx, e_out, g_out, pairs, cg.MODE_PLAIN if mode is None else mode, step, P, F)
        st = cg.compton_get_stats(ctx, reset=True)
        off_e = _dev_array(torch, pairs.off_e_dev, w.n_cells + 1).astype(np.int64)
        off_g = _dev_array(torch, pairs.off_g_dev, w.n_cells + 1).astype(np.int64)
        np_ = int(st["pairs_tested"])
        return dict(be=be, bg=bg, ae=species_np(e_out), ag=species_np(g_out),
                    P=None if P is None else P.cpu().numpy()[:np_].astype(np.float64),
                    F=F.cpu().numpy()[:np_], off_e=off_e, off_g=off_g, n=np_, stats=st)
    finally:
        cg.compton_destroy(ctx)


def _pairs(off_e, off_g, n_cells):
    m = np.minimum(np.diff(off_e), np.diff(off_g))
    cell = np.repeat(np.arange(n_cells), m)
    j = np.arange(cell.shape[0]) - np.concatenate([[0], np.cumsum(m)])[cell]
    return off_e[cell] + j, off_g[cell] + j, cell


@pytest.mark.parametrize("seed,both", [(21, True), (22, False)])
def test_weighted_step_matches_oracle(seed, both):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w, e, g = _weighted(seed, both)
    step = 5
    r = _run(cg, torch, w, e, g, step)
    o = oracle.step_weighted(w.n_cells, w.w_over_v, w.dt, w.seed, step, e, g)
    # binning: order, offsets and the weights that travel along, bit-exact
    assert np.array_equal(r["be"]["id"], e["id"][o["e_perm"]])
    assert np.array_equal(r["bg"]["id"], g["id"][o["g_perm"]])
    assert np.array_equal(r["off_e"], o["e_off"]) and np.array_equal(r["off_g"], o["g_off"])
    assert np.array_equal(r["be"]["w"].astype(np.float64), o["e_w"])
    if both:
        assert np.array_equal(r["bg"]["w"].astype(np.float64), o["g_w"])
    assert np.array_equal(r["ae"]["w"], r["be"]["w"])  # the step leaves weights alone
    n = o["n_pairs"]
    assert r["n"] == n
    assert np.allclose(r["P"], o["P"], rtol=2e-5, atol=1e-9)
    u0 = u0_of_pairs(w.seed, step, n)
    near = np.abs(u0 - o["P"]) < FLIP_BAND
    assert np.array_equal(r["F"][~near], o["flag"][~near])
    ok = (r["F"] == o["flag"])
    ie, ig, _ = _pairs(r["off_e"], r["off_g"], w.n_cells)
    ub, kb = _mom(r["be"]), _mom(r["bg"])
    ua, ka = _mom(r["ae"]), _mom(r["ag"])
    # which partner took its new momentum: compare with the oracle's upd bits
    moved_e = np.any(ua[:, ie] != ub[:, ie], axis=0)
    moved_g = np.any(ka[:, ig] != kb[:, ig], axis=0)
    hit = ok & (o["flag"] == 1)
    assert hit.sum() > 100
    rej_e = hit & ((o["upd"] & 1) == 0)
    rej_g = hit & ((o["upd"] & 2) == 0)
    assert rej_e.sum() + rej_g.sum() > 20  # the rejection path is exercised
    assert not np.any(moved_e[rej_e]) and not np.any(moved_g[rej_g])
    scale = energy_scale(ub[:, ie], kb[:, ig])
    du = np.linalg.norm(ua[:, ie] - o["e_out"][:, ie], axis=0)
    dk = np.linalg.norm(ka[:, ig] - o["g_out"][:, ig], axis=0)
    assert np.all(du[ok] <= MOM_TOL * scale[ok]), np.max(du[ok] / scale[ok])
    assert np.all(dk[ok] <= MOM_TOL * scale[ok]), np.max(dk[ok] / scale[ok])
    assert r["stats"]["scatters"] == int(r["F"].sum())


def test_weighted_pnet_mode_uses_the_pair_weights():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w, e, g = _weighted(23)
    th = opn.init_params(14)
    th[opn.N_PARAMS - 1] = -1.0
    th32 = th.astype(np.float32)
    r = _run(cg, torch, w, e, g, 1, mode=cg.MODE_PNET, th=th32)
    ie, ig, cell = _pairs(r["off_e"], r["off_g"], w.n_cells)
    nmax = np.maximum(np.diff(r["off_e"]), np.diff(r["off_g"]))[cell].astype(np.float32)
    we, wg = r["be"]["w"][ie], r["bg"]["w"][ig]
    dens = (nmax * np.maximum(we, wg)).astype(np.float32).astype(np.float64)
    u, k = _mom(r["be"])[:, ie], _mom(r["bg"])[:, ig]
    g2 = 1.0 + (u ** 2).sum(0)
    e2 = (k ** 2).sum(0)
    inr = (g2 <= 1e6) & (e2 >= 1e-8) & (e2 <= 1.0) & (r["P"] > 1e-6) & (r["P"] < 0.5)
    assert inr.sum() > 1000
    f = opn.features(u, k, we.astype(np.float64), wg.astype(np.float64), 2.0 * dens * w.dt)
    r_ref, _ = opn.forward(th32.astype(np.float64), f)
    # the network output behind each P (FP32 P: relative error ~1e-7)
    r_gpu = -np.log1p(-r["P"]) / (2.0 * dens * w.dt)
    assert np.all(np.abs(r_gpu[inr] - r_ref[inr]) <= 5e-6 + 1e-5 * r_ref[inr])


@pytest.mark.parametrize("mode_name", ["MODE_PLAIN", "MODE_MLP_BF16", "MODE_PNET"])
def test_weighted_filtered_equals_full_evaluation(mode_name):
    # without prob_out only pairs below their own bound 1 - exp(-2 n_p dt)
    # are evaluated; the outcome is that of evaluating every pair
    import paper_2206_02937_gb300 as cg
    from oracle import mlp as omlp
    torch = torch_cuda()
    cg.build()
    mode = getattr(cg, mode_name)
    w, e, g = _weighted(25)
    outs = []
    for want_p in (True, False):
        ctx_th = opn.init_params(15).astype(np.float32) if mode == cg.MODE_PNET else None
        if mode == cg.MODE_MLP_BF16:
            ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
            try:
                cg.compton_mlp_set_params(ctx, omlp.init_params(9).astype(np.float32))
                e_in, g_in = to_species(torch, e), to_species(torch, g)
                e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
                pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 4)
                F = torch.zeros(pairs.max_pairs, dtype=torch.uint8, device="cuda")
                P = torch.zeros(pairs.max_pairs, device="cuda") if want_p else None
                cg.compton_scatter_step(ctx, e_out, g_out, pairs, mode, 4, P, F)
                outs.append(dict(ae=species_np(e_out), ag=species_np(g_out), F=F.cpu().numpy()))
            finally:
                cg.compton_destroy(ctx)
        else:
            outs.append(_run(cg, torch, w, e, g, 4, mode=mode, th=ctx_th, want_p=want_p))
    a, b = outs
    assert a["F"].sum() > 20
    assert np.array_equal(a["F"], b["F"])
    for c in ("ux", "uy", "uz"):
        assert np.array_equal(a["ae"][c], b["ae"][c]) and np.array_equal(a["ag"][c], b["ag"][c])


def test_weight_argument_checks():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w, e, g = _weighted(24, nx=8, ppc=8)
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        e_in, g_in = to_species(torch, e), to_species(torch, g)
        e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
        bare = cg.Species(e_out.ux, e_out.uy, e_out.uz, e_out.cell, e_out.id)
        with pytest.raises(cg.ComptonError):  # weighted input, no output weights
            cg.compton_bin_pairs(ctx, e_in, g_in, bare, g_out, 0)
        pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 0)
        with pytest.raises(cg.ComptonError):  # binned with weights, scattered without
            cg.compton_scatter_step(ctx, bare, cg.Species(g_out.ux, g_out.uy, g_out.uz, g_out.cell, g_out.id),
                                    pairs, cg.MODE_PLAIN, 0)
        with pytest.raises(cg.ComptonError):  # No-Time-Counter takes equal weights only
            cg.compton_scatter_step_ntc(ctx, e_out, g_out, pairs, 0)
        cg.compton_scatter_step(ctx, e_out, g_out, pairs, cg.MODE_PLAIN, 0)
        torch.cuda.synchronize()
    finally:
        cg.compton_destroy(ctx)
