"""The paper's own 9-12-9 network (Sec. 3.2, Fig. 2a) on the GPU against the
FP64 oracle: inference, gradient and Adam step, learning of the analytic
ratio, and the scatter step in COMPTON_MODE_PNET."""
import numpy as np
import pytest

import oracle
from oracle import pnet as opn
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import _dev_array, energy_scale, species_np, to_species, torch_cuda

pytestmark = pytest.mark.gpu

W_E, W_G, P_MAX = 0.01, 0.02, 0.3


def _ctx(cg, batch):
    return cg.compton_init(1, 0, 1.0, 0.05, 1, max_train_batch=batch)


def _cuda(torch, *arrays):
    return tuple(None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
                 for a in arrays)


@pytest.mark.parametrize("n", [1, 1000, 70001])
def test_inference_matches_oracle(n):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    u, k = wl.c3(n, seed=71)
    th = opn.init_params(3)
    th[opn.N_PARAMS - 1] = -2.0  # output bias: r spread over (0, 1)
    th32 = th.astype(np.float32)
    ctx = _ctx(cg, 16)
    try:
        cg.compton_pnet_set_params(ctx, th32)
        ut, kt = _cuda(torch, u, k)
        r = torch.zeros(n, device="cuda")
        cg.compton_pnet_infer(ctx, ut, kt, W_E, W_G, P_MAX, r)
        r = r.cpu().numpy().astype(np.float64)
    finally:
        cg.compton_destroy(ctx)
    f = opn.features(u.astype(np.float64), k.astype(np.float64), W_E, W_G, P_MAX)
    r_ref, _ = opn.forward(th32.astype(np.float64), f)
    # FP32 features and four FP32 layers: absolute error a few 1e-7
    assert np.max(np.abs(r - r_ref)) <= 5e-6


@pytest.mark.parametrize("n,weighted", [(1000, False), (4097, True)])
def test_gradient_and_adam_match_oracle(n, weighted):
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    u, k = wl.c3(n, seed=72)
    rng = np.random.default_rng(73)
    y = rng.uniform(0.02, 0.98, n)
    w = rng.uniform(0.5, 2.0, n) if weighted else None
    th32 = opn.init_params(8).astype(np.float32)
    lr = 1e-3
    ctx = _ctx(cg, n)
    try:
        cg.compton_pnet_set_params(ctx, th32)
        ut, kt, yt, wt = _cuda(torch, u, k, y, w)
        loss = cg.compton_pnet_train_step(ctx, ut, kt, yt, wt, W_E, W_G, P_MAX, lr=lr)
        th_new, g_gpu = (a.astype(np.float64) for a in cg.compton_pnet_get_params(ctx))
    finally:
        cg.compton_destroy(ctx)
    th64 = th32.astype(np.float64)
    f = opn.features(u.astype(np.float64), k.astype(np.float64), W_E, W_G, P_MAX)
    loss_ref, g_ref = opn.backward(th64, f, y.astype(np.float32).astype(np.float64),
                                   None if w is None else w.astype(np.float32).astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    for (Wg, bg), (Wr, br) in zip(opn.unpack(g_gpu), opn.unpack(g_ref)):
        assert np.linalg.norm(Wg - Wr) <= 1e-4 * np.linalg.norm(Wr) + 1e-9
        assert np.linalg.norm(bg - br) <= 1e-4 * np.linalg.norm(br) + 1e-9
    # first Adam step (Kingma and Ba 2014): m_hat = g, v_hat = g^2, so the
    # update is lr g / (|g| + 1e-7) from the oracle's own gradient; where the
    # gradient is well above its FP32 noise the two updates agree closely,
    # elsewhere the update is still bounded by lr
    step_ref = -lr * g_ref / (np.abs(g_ref) + 1e-7)
    step_gpu = th_new - th64
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    assert big.sum() > 0.5 * big.size
    assert np.allclose(step_gpu[big], step_ref[big], rtol=1e-3, atol=1e-9)
    assert np.all(np.abs(step_gpu) <= lr * (1.0 + 1e-5) + 1e-7 * np.abs(th64))


def test_training_learns_the_analytic_ratio():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    n_train, n_test, batch = 65536, 8192, 4096
    u, k = wl.c3(n_train + n_test, seed=74)
    ctx = _ctx(cg, batch)
    try:
        ut, kt = _cuda(torch, u, k)
        r = torch.zeros(n_train + n_test, device="cuda")
        cg.compton_kn_ratio(ctx, ut, kt, r)
        cg.compton_pnet_set_params(ctx, opn.init_params(5).astype(np.float32))
        te = slice(n_train, None)
        r_hat = torch.zeros(n_test, device="cuda")

        def test_mae():
            cg.compton_pnet_infer(ctx, ut[:, te].contiguous(), kt[:, te].contiguous(), W_E, W_G, P_MAX, r_hat)
            torch.cuda.synchronize()
            return float((r_hat - r[te]).abs().mean())

        mae0 = test_mae()
        losses = []
        gen = torch.Generator(device="cuda").manual_seed(0)
        for it in range(600):
            idx = torch.randint(0, n_train, (batch,), device="cuda", generator=gen)
            losses.append(cg.compton_pnet_train_step(ctx, ut[:, idx].contiguous(), kt[:, idx].contiguous(),
                                                     r[idx].contiguous(), None, W_E, W_G, P_MAX, lr=1e-2,
                                                     want_loss=(it % 50 == 0)))
        mae1 = test_mae()
    finally:
        cg.compton_destroy(ctx)
    ls = [l_ for l_ in losses if l_ is not None]
    assert ls[-1] < 0.5 * ls[0]
    assert mae1 < 0.5 * mae0, (mae0, mae1)


def test_set_params_rejects_bad_arguments():
    import paper_2206_02937_gb300 as cg
    torch_cuda()
    cg.build()
    ctx = _ctx(cg, 16)
    try:
        th = opn.init_params(1).astype(np.float32)
        with pytest.raises(cg.ComptonError):
            cg.compton_pnet_set_params(ctx, th[:-1])
        with pytest.raises(cg.ComptonError):
            cg.compton_pnet_set_params(ctx, th, feature_scales=[1.0, 0.0, 1.0, 1.0])
        with pytest.raises(cg.ComptonError):
            cg.compton_pnet_set_params(ctx, th, eps_min=1.0, eps_max=0.5)
        with pytest.raises(cg.ComptonError):  # no network loaded yet
            cg.compton_pnet_get_params(ctx)
    finally:
        cg.compton_destroy(ctx)


def _scatter_workload(seed):
    w = wl.c2(48, 48, 40, seed=seed)
    rng = wl.rng_for(seed + 50)
    # some pairs outside the training range: gamma > 1e3, eps < 1e-4, eps > 1
    for frac, scale, sp in ((0.02, 3e3, w.e), (0.02, 3e-3, w.g), (0.01, 300.0, w.g)):
        idx = rng.choice(sp["ux"].shape[0], int(frac * sp["ux"].shape[0]), replace=False)
        for c in ("ux", "uy", "uz"):
            sp[c][idx] = (sp[c][idx] * scale).astype(np.float32)
    return w


def test_scatter_step_in_pnet_mode():
    # in-range pairs take P = 1 - exp(-2 n dt r) with r the network's (the
    # inference entry point on the same pair, weights w/V, P_max = 2 n dt);
    # the others the analytic probability; collisions follow the oracle
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w = _scatter_workload(5)
    th = opn.init_params(12)
    th[opn.N_PARAMS - 1] = -1.0
    th32 = th.astype(np.float32)
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        cg.compton_pnet_set_params(ctx, th32)
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
        u = np.stack([be[c][ie] for c in ("ux", "uy", "uz")]).astype(np.float32)
        k = np.stack([bg[c][ig] for c in ("ux", "uy", "uz")]).astype(np.float32)
        dens32 = (np.maximum(np.diff(off_e), np.diff(off_g))[cell] * np.float32(w.w_over_v)).astype(np.float32)
        r = np.zeros(n)
        for d in np.unique(dens32):
            sel = np.nonzero(dens32 == d)[0]
            rt = torch.zeros(sel.size, device="cuda")
            ut, kt = _cuda(torch, u[:, sel], k[:, sel])
            p_max = float(np.float32(2.0) * d * np.float32(w.dt))
            cg.compton_pnet_infer(ctx, ut, kt, w.w_over_v, w.w_over_v, p_max, rt)
            r[sel] = rt.cpu().numpy()
        P = torch.zeros(n, device="cuda")
        F = torch.zeros(n, dtype=torch.uint8, device="cuda")
        cg.compton_get_stats(ctx, reset=True)
        cg.compton_scatter_step(ctx, e_out, g_out, pairs, cg.MODE_PNET, 0, P, F)
        st = cg.compton_get_stats(ctx, reset=True)
        ae, ag = species_np(e_out), species_np(g_out)
        P, F = P.cpu().numpy().astype(np.float64), F.cpu().numpy()
    finally:
        cg.compton_destroy(ctx)
    dens = dens32.astype(np.float64)
    g2 = 1.0 + (u.astype(np.float64) ** 2).sum(0)
    e2 = (k.astype(np.float64) ** 2).sum(0)
    in_range = (g2 <= 1e6) & (e2 >= 1e-8) & (e2 <= 1.0)
    assert st["mlp_fallbacks"] == int((~in_range).sum()) > 0
    # the network's r itself is pinned to the oracle by the inference test
    f = opn.features(u.astype(np.float64), k.astype(np.float64), w.w_over_v, w.w_over_v, 2.0 * dens * w.dt)
    r_ref, _ = opn.forward(th32.astype(np.float64), f)
    assert np.max(np.abs(r - r_ref)) <= 5e-6
    P_net = 1.0 - np.exp(-2.0 * dens * w.dt * r)
    assert np.allclose(P[in_range], P_net[in_range], rtol=1e-5, atol=1e-9)
    P_ana = np.array([oracle.scatter_event(u[:, q], k[:, q], dens[q], w.dt, w.seed, 0, q)[2]
                      for q in np.nonzero(~in_range)[0]])
    assert np.allclose(P[~in_range], P_ana, rtol=2e-5, atol=1e-9)
    u0 = np.array([oracle.bernoulli_u0(w.seed, 0, q) for q in range(n)])
    assert np.array_equal(F, (u0 < P).astype(np.uint8))
    hit = np.nonzero(F)[0]
    assert hit.size > 50 and st["scatters"] == hit.size
    scale = energy_scale(u, k)
    for q in hit[:400]:
        uo, ko = oracle.collide(u[:, q].astype(np.float64), k[:, q].astype(np.float64), w.seed, 0, int(q))
        ua = np.array([ae[c][ie[q]] for c in ("ux", "uy", "uz")], dtype=np.float64)
        ka = np.array([ag[c][ig[q]] for c in ("ux", "uy", "uz")], dtype=np.float64)
        assert np.linalg.norm(ua - uo) <= 1e-5 * scale[q]
        assert np.linalg.norm(ka - ko) <= 1e-5 * scale[q]


def test_pnet_mode_filtered_equals_full_evaluation():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w = _scatter_workload(6)
    th = opn.init_params(13)
    th[opn.N_PARAMS - 1] = -1.0
    out = {}
    for want_p in (True, False):
        ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
        try:
            cg.compton_pnet_set_params(ctx, th.astype(np.float32))
            e_in, g_in = to_species(torch, w.e), to_species(torch, w.g)
            e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
            pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 2)
            n = pairs.max_pairs
            P = torch.zeros(n, device="cuda") if want_p else None
            F = torch.zeros(n, dtype=torch.uint8, device="cuda")
            cg.compton_get_stats(ctx, reset=True)
            cg.compton_scatter_step(ctx, e_out, g_out, pairs, cg.MODE_PNET, 2, P, F)
            st = cg.compton_get_stats(ctx, reset=True)
            out[want_p] = (F.cpu().numpy(), species_np(e_out), species_np(g_out), st)
        finally:
            cg.compton_destroy(ctx)
    (Fa, ea, ga, sa), (Fb, eb, gb, sb) = out[True], out[False]
    assert np.array_equal(Fa, Fb) and Fa.sum() > 20
    assert sa["scatters"] == sb["scatters"]
    for c in ("ux", "uy", "uz"):
        assert np.array_equal(ea[c], eb[c]) and np.array_equal(ga[c], gb[c])


def test_pnet_mode_needs_parameters():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w = wl.c2(8, 8, 4, seed=1)
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        e_in, g_in = to_species(torch, w.e), to_species(torch, w.g)
        e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
        pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 0)
        with pytest.raises(cg.ComptonError):
            cg.compton_scatter_step(ctx, e_out, g_out, pairs, cg.MODE_PNET, 0)
    finally:
        cg.compton_destroy(ctx)
