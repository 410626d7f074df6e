"""Parity of the CUDA path (bin_pairs + scatter_step through the C ABI) with
the FP64 oracle, element by element on seeded inputs.

Tolerances (the benchmark spec of the method's parity):
  * pairing order, cell offsets, pair count: bit-exact;
  * Bernoulli decisions: bit-exact except where |u0 - P_oracle| < 1e-6;
  * momenta: |du| and |dk| <= 1e-5 (gamma + eps) of the pair, FP32 storage;
  * untouched particles: bit-exact copies.
"""
import numpy as np
import pytest

import oracle
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import energy_scale, gpu_step, u0_of_pairs

pytestmark = pytest.mark.gpu

FLIP_BAND = 1e-6
MOM_TOL = 1e-5


def _pair_index(off_e, off_g, n_cells):
    ce = np.diff(off_e.astype(np.int64))
    cg = np.diff(off_g.astype(np.int64))
    m = np.minimum(ce, cg)
    pair_cell = np.repeat(np.arange(n_cells), m)
    pair_off = np.concatenate([[0], np.cumsum(m)])
    j = np.arange(pair_cell.shape[0]) - pair_off[pair_cell]
    return off_e[pair_cell] + j, off_g[pair_cell] + j, pair_cell


def _mom(s):
    return np.stack([s["ux"], s["uy"], s["uz"]]).astype(np.float64)


def compare_with_oracle(w, step=0, gamma64=1.0e3):
    g = gpu_step(w, step=step, gamma64=gamma64)
    o = oracle.step(w.n_cells, w.w_over_v, w.dt, w.seed, step, w.e, w.g)
    assert g["check"] == 0
    # ordering and offsets: bit-exact
    assert np.array_equal(g["before_e"]["id"], w.e["id"][o["e_perm"]])
    assert np.array_equal(g["before_g"]["id"], w.g["id"][o["g_perm"]])
    assert np.array_equal(g["before_e"]["cell"], w.e["cell"][o["e_perm"]])
    assert np.array_equal(g["off_e"], o["e_off"])
    assert np.array_equal(g["off_g"], o["g_off"])
    assert g["n_pairs"] == o["n_pairs"]
    n = o["n_pairs"]
    if n == 0:
        assert np.array_equal(g["after_e"]["ux"], g["before_e"]["ux"])
        return g, o, 0
    # probabilities (FP32 vs FP64) and decisions
    assert np.allclose(g["P"], o["P"], rtol=2e-5, atol=1e-9)
    u0 = u0_of_pairs(w.seed, step, n)
    near = np.abs(u0 - o["P"]) < FLIP_BAND
    assert np.array_equal(g["flag"][~near], o["flag"][~near])
    flips = np.nonzero(g["flag"] != o["flag"])[0]
    # momenta, per particle, against the pair's energy scale
    ie, ig, _ = _pair_index(g["off_e"], g["off_g"], w.n_cells)
    ue_b, kg_b = _mom(g["before_e"]), _mom(g["before_g"])
    scale = energy_scale(ue_b[:, ie], kg_b[:, ig])
    du = np.linalg.norm(_mom(g["after_e"])[:, ie] - o["e_out"][:, ie], axis=0)
    dk = np.linalg.norm(_mom(g["after_g"])[:, ig] - o["g_out"][:, ig], axis=0)
    ok = np.ones(n, dtype=bool)
    ok[flips] = False
    assert np.all(du[ok] <= MOM_TOL * scale[ok]), np.max(du[ok] / scale[ok])
    assert np.all(dk[ok] <= MOM_TOL * scale[ok]), np.max(dk[ok] / scale[ok])
    # unpaired particles are untouched
    paired_e = np.zeros(w.n_e, dtype=bool)
    paired_e[ie] = True
    assert np.array_equal(g["after_e"]["ux"][~paired_e], g["before_e"]["ux"][~paired_e])
    # unscattered pairs are untouched (bit-exact)
    still = (g["flag"] == 0)
    assert np.array_equal(g["after_e"]["uy"][ie[still]], g["before_e"]["uy"][ie[still]])
    assert np.array_equal(g["after_g"]["uz"][ig[still]], g["before_g"]["uz"][ig[still]])
    # energy-momentum conservation of the GPU's own scattered pairs
    hit = np.nonzero(g["flag"] == 1)[0]
    if hit.size:
        ua, ka = _mom(g["after_e"])[:, ie[hit]], _mom(g["after_g"])[:, ig[hit]]
        ub, kb = ue_b[:, ie[hit]], kg_b[:, ig[hit]]
        Eb = energy_scale(ub, kb)
        Ea = energy_scale(ua, ka)
        assert np.all(np.abs(Ea - Eb) <= 2e-6 * Eb)
        assert np.all(np.linalg.norm((ua + ka) - (ub + kb), axis=0) <= 2e-6 * Eb)
    return g, o, len(flips)


def test_c1_full():
    w = wl.c1()
    g, o, flips = compare_with_oracle(w)
    assert o["n_pairs"] == 4096
    # about 0.05 <s v> of the pairs collide (P ~ n dt s v with n = 1, dt = 0.05)
    assert 120 < o["flag"].sum() < 300
    assert flips <= 2


def _random_workload(seed, n_cells, ppc_e, ppc_g, spread=0.5, gamma_max=100.0, eps=(1e-4, 1.0)):
    rng = wl.rng_for(seed)
    ce = wl.lognormal_counts(rng, n_cells, ppc_e, spread)
    cg = wl.lognormal_counts(rng, n_cells, ppc_g, spread)
    ce[rng.uniform(size=n_cells) < 0.05] = 0  # some cells without electrons
    cg[rng.uniform(size=n_cells) < 0.05] = 0  # some without photons
    cell_e = rng.permutation(np.repeat(np.arange(n_cells), ce))
    cell_g = rng.permutation(np.repeat(np.arange(n_cells), cg))
    ne, ng = cell_e.shape[0], cell_g.shape[0]
    gam = 10 ** rng.uniform(0, np.log10(gamma_max), ne)
    u = np.sqrt(gam ** 2 - 1) * wl.isotropic(rng, ne)
    k = 10 ** rng.uniform(np.log10(eps[0]), np.log10(eps[1]), ng) * wl.isotropic(rng, ng)
    e = wl._species(u, cell_e)
    g = wl._species(k, cell_g)
    e["id"] = rng.permutation(3 * ne)[:ne].astype(np.uint32)  # sparse unique ids
    g["id"] = rng.permutation(3 * ng)[:ng].astype(np.uint32)
    return wl.Workload(f"random {seed}", n_cells, 2.0 / max(ppc_e, 1), 0.05, 1000 + seed, 1, e, g)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_ragged(seed):
    # several scatter tiles (1024 pairs) and sort tiles (512 particles), ragged tails
    w = _random_workload(seed, n_cells=257 + 37 * seed, ppc_e=40 + 7 * seed, ppc_g=33)
    compare_with_oracle(w, step=seed)


def test_step_and_seed_high_words():
    w = _random_workload(4, 50, 30, 30)
    w.seed = (7 << 32) + 3
    compare_with_oracle(w, step=(1 << 32) + 11)


def test_large_gamma_fp32_matches_fp64_branch():
    # electrons up to gamma 1e5, nearly collinear photons: the FP32 invariants
    # alone (threshold inf) and the FP64 branch (threshold 0) both hold parity
    w = _random_workload(5, 64, 32, 32, gamma_max=1e5, eps=(1e-4, 1e-2))
    compare_with_oracle(w, gamma64=float("inf"))
    compare_with_oracle(w, gamma64=0.0)


def test_cells_larger_than_shared_tile():
    # cells of 3000 particles: a sort tile's cell range exceeds shared memory
    w = _random_workload(6, 5, 3000, 2800, spread=0.05)
    compare_with_oracle(w)


def test_single_giant_cell():
    # one cell above the shared-memory capacity takes the global-memory path
    rng = wl.rng_for(7)
    n = 7000
    u = 3.0 * wl.isotropic(rng, n)
    k = 0.01 * wl.isotropic(rng, n)
    cell = np.zeros(n, dtype=np.int64)
    w = wl.Workload("giant", 3, 1.0 / 5000, 0.05, 9, 1, wl._species(u, cell), wl._species(k, cell))
    compare_with_oracle(w)


def test_empty_and_one_sided():
    rng = wl.rng_for(8)
    u = wl.isotropic(rng, 100)
    e = wl._species(u, np.arange(100) % 10)
    g = wl._species(np.zeros((3, 0)), np.zeros(0, dtype=np.int64))
    w = wl.Workload("no photons", 10, 0.1, 0.05, 1, 1, e, g)
    g_, o, _ = compare_with_oracle(w)
    assert o["n_pairs"] == 0
    # photons only in cells without electrons
    g2 = wl._species(0.1 * wl.isotropic(rng, 50), 10 + np.arange(50) % 5)
    w2 = wl.Workload("disjoint", 15, 0.1, 0.05, 1, 1, e, g2)
    _, o2, _ = compare_with_oracle(w2)
    assert o2["n_pairs"] == 0


def test_cell_out_of_range_reported():
    import paper_2206_02937_gb300 as cgl
    from tests.gpu_util import to_species, torch_cuda
    torch = torch_cuda()
    rng = wl.rng_for(9)
    e = wl._species(wl.isotropic(rng, 64), np.arange(64) % 8)
    g = wl._species(wl.isotropic(rng, 64), np.arange(64) % 8)
    e["cell"][5] = 8  # one past the last cell
    cgl.build()
    ctx = cgl.compton_init(8, 64, 0.1, 0.05, 1)
    try:
        ei, gi = to_species(torch, e), to_species(torch, g)
        eo, go = cgl.Species.empty_like(ei), cgl.Species.empty_like(gi)
        cgl.compton_bin_pairs(ctx, ei, gi, eo, go, 0)
        assert cgl.compton_check(ctx) == cgl.COMPTON_ERANGE
        assert cgl.compton_check(ctx) == cgl.COMPTON_OK  # cleared
    finally:
        cgl.compton_destroy(ctx)


def test_explicit_pairs_and_ratio():
    import paper_2206_02937_gb300 as cgl
    from tests.gpu_util import torch_cuda
    torch = torch_cuda()
    cgl.build()
    u, k = wl.c3(5000, seed=11)
    nd = np.full(5000, 20.0, dtype=np.float32)
    uo, ko, P, flag = oracle.pairs(u, k, nd, 0.05, 77, 4)
    r_or = oracle.ratio(u, k)
    ctx = cgl.compton_init(1, 0, 1.0, 0.05, 1)
    try:
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        r = torch.zeros(5000, device="cuda")
        cgl.compton_kn_ratio(ctx, ut, kt, r)
        assert np.allclose(r.cpu().numpy(), r_or, rtol=2e-5, atol=1e-12)
        Pg = torch.zeros(5000, device="cuda")
        fg = torch.zeros(5000, dtype=torch.uint8, device="cuda")
        cgl.compton_scatter_pairs(ctx, ut, kt, torch.from_numpy(nd).cuda(), 77, 4, cgl.MODE_PLAIN, Pg, fg)
        torch.cuda.synchronize()
        assert np.allclose(Pg.cpu().numpy(), P, rtol=2e-5, atol=1e-9)
        u0 = u0_of_pairs(77, 4, 5000)
        near = np.abs(u0 - P) < FLIP_BAND
        fgn = fg.cpu().numpy()
        assert np.array_equal(fgn[~near], flag[~near])
        ok = fgn == flag
        scale = energy_scale(u, k)
        du = np.linalg.norm(ut.cpu().numpy().astype(np.float64) - uo, axis=0)
        dk = np.linalg.norm(kt.cpu().numpy().astype(np.float64) - ko, axis=0)
        assert np.all(du[ok] <= MOM_TOL * scale[ok]) and np.all(dk[ok] <= MOM_TOL * scale[ok])
        assert flag.sum() > 100
    finally:
        cgl.compton_destroy(ctx)


def _presorted(w):
    """The same particles, stably ordered by cell: the binning then reads the
    input in place instead of placing records first."""
    out = wl.Workload(w.name + " presorted", w.n_cells, w.w_over_v, w.dt, w.seed, w.steps)
    for name in ("e", "g"):
        sp = getattr(w, name)
        order = np.argsort(sp["cell"], kind="stable")
        setattr(out, name, {k: np.ascontiguousarray(v[order]) for k, v in sp.items()})
    return out


@pytest.mark.parametrize("case", ["ragged", "big_cells", "one_sided"])
def test_presorted_input(case):
    if case == "ragged":
        w = _random_workload(12, n_cells=601, ppc_e=45, ppc_g=38)
    elif case == "big_cells":
        w = _random_workload(13, 6, 3000, 2800, spread=0.05)  # tiles above shared memory, cells above it too
    else:
        rng = wl.rng_for(14)
        e = wl._species(wl.isotropic(rng, 300), np.arange(300) % 30)
        g = wl._species(0.1 * wl.isotropic(rng, 90), 3 * (np.arange(90) % 10))
        w = wl.Workload("one-sided", 40, 0.1, 0.05, 5, 1, e, g)
    compare_with_oracle(_presorted(w), step=3)


def test_two_chained_steps():
    # the sorted output of one step is the next step's input (the in-place
    # path); the oracle's second step starts from the GPU's first-step output
    w = _random_workload(15, n_cells=333, ppc_e=50, ppc_g=47)
    g1, _, _ = compare_with_oracle(w, step=0)
    w2 = wl.Workload("second step", w.n_cells, w.w_over_v, w.dt, w.seed, 1,
                     {k: np.ascontiguousarray(v) for k, v in g1["after_e"].items()},
                     {k: np.ascontiguousarray(v) for k, v in g1["after_g"].items()})
    compare_with_oracle(w2, step=1)


def test_unaligned_input_arrays():
    # species arrays that start 4 bytes past an aligned address (views at
    # offset 1): the histogram and the sort's staging take their scalar
    # loads; order and momenta must match
    import paper_2206_02937_gb300 as cgl
    from tests.gpu_util import species_np, torch_cuda
    torch = torch_cuda()
    cgl.build()
    w = _presorted(_random_workload(16, n_cells=129, ppc_e=21, ppc_g=19))

    def shifted(d):
        def t(a):
            base = torch.zeros(a.shape[0] + 1, dtype=torch.from_numpy(a).dtype, device="cuda")
            base[1:] = torch.from_numpy(a).cuda()
            return base[1:]
        return cgl.Species(t(d["ux"]), t(d["uy"]), t(d["uz"]), t(d["cell"]), t(d["id"].view(np.int32)))

    o = oracle.step(w.n_cells, w.w_over_v, w.dt, w.seed, 2, w.e, w.g)
    ctx = cgl.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        e_in, g_in = shifted(w.e), shifted(w.g)
        assert e_in.cell.data_ptr() % 16 != 0
        e_out, g_out = cgl.Species.empty_like(e_in), cgl.Species.empty_like(g_in)
        cgl.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 2)
        torch.cuda.synchronize()
        assert cgl.compton_check(ctx) == cgl.COMPTON_OK
        be, bg = species_np(e_out), species_np(g_out)
    finally:
        cgl.compton_destroy(ctx)
    assert np.array_equal(be["id"], w.e["id"][o["e_perm"]])
    assert np.array_equal(bg["id"], w.g["id"][o["g_perm"]])
    for c in ("ux", "uy", "uz"):
        assert np.array_equal(be[c], w.e[c][o["e_perm"]])
        assert np.array_equal(bg[c], w.g[c][o["g_perm"]])


@pytest.mark.parametrize("case", ["c1", "ragged", "gamma_fp64", "gamma_fp32"])
def test_filtered_equals_full_evaluation(case):
    # without prob_out only pairs whose uniform lies below the bound
    # 1 - exp(-2 n dt) are evaluated; decisions and momenta must be those of
    # the full evaluation (which the tests above hold to the oracle)
    gamma64 = 1.0e3
    if case == "c1":
        w = wl.c1()
    elif case == "ragged":
        w = _random_workload(17, n_cells=700, ppc_e=44, ppc_g=40)
    else:
        w = _random_workload(18, 64, 32, 32, gamma_max=1e5, eps=(1e-4, 1e-2))
        gamma64 = 0.0 if case == "gamma_fp64" else float("inf")
    full = gpu_step(w, step=5, gamma64=gamma64)
    flt = gpu_step(w, step=5, gamma64=gamma64, want_prob=False, want_flag=True)
    bare = gpu_step(w, step=5, gamma64=gamma64, want_prob=False)
    assert np.array_equal(flt["flag"], full["flag"])
    assert flt["stats"]["scatters"] == full["stats"]["scatters"] == bare["stats"]["scatters"]
    for g in (flt, bare):
        for sp in ("after_e", "after_g"):
            for c in ("ux", "uy", "uz"):
                assert np.array_equal(g[sp][c], full[sp][c])


@pytest.mark.parametrize("presorted", [False, True])
def test_tiles_above_shared_memory_in_chunks(presorted):
    # cells of ~700 particles (spread 0.3): sort tiles above shared memory,
    # sorted in runs of whole cells that fit, and cells above it alone, ranked
    # in global memory
    w = _random_workload(19, 40, 700, 650, spread=0.3)
    compare_with_oracle(_presorted(w) if presorted else w, step=4)


def test_sparse_cells_beyond_the_staged_window():
    # about one particle of each species per cell, many cells empty: each
    # tile of 1024 pairs spans about 2000 cells, more than the probability
    # kernel stages in shared memory (512), so its cell records are read
    # from global memory
    w = _random_workload(21, n_cells=12000, ppc_e=1, ppc_g=1, spread=0.8)
    g, o, _ = compare_with_oracle(w, step=3)
    assert o["n_pairs"] > 2048
