"""Oracle parity of the exact configuration bench.py times.

Every timed step of the benchmark bins the previous step's output, which is
already in cell order (the in-place sort path of compton_bin_pairs), and calls
compton_scatter_step with neither probabilities nor flags requested, so that
only the pairs below the probability bound are evaluated (the filtered path of
the scatter kernel).  These tests run that chain: step 0 bins shuffled input,
step 1 bins step 0's output, both through the benchmark's calls, and step 1
is compared with the FP64 oracle (Sec. 3.1: pairing in each cell, a random
number against the probability, the collision of accepted pairs).

* 256 x 256 cells (4.2M pairs, about 4000 scatter tiles, far more than the
  persistent CTAs, so every CTA takes many tiles with the filter on): the
  whole step against the oracle's step, pair by pair.
* 512 x 512 cells (16.8M pairs, the benchmark's size): offsets of every
  cell, the sorted order of sampled cells against the oracle's sort, sampled
  pairs and every
  collision among the first 2000 pairs against the oracle's event, and the
  timed call's result equal, bit for bit, to the same step with every pair's
  probability and flag requested.
"""
import numpy as np
import pytest

import oracle
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import _dev_array, energy_scale, species_np, to_species, torch_cuda

pytestmark = pytest.mark.gpu

MOM = ("ux", "uy", "uz")


def _mom(s, idx=None):
    if idx is None:
        return np.stack([s[a] for a in MOM]).astype(np.float64)
    return np.stack([s[a][idx] for a in MOM]).astype(np.float64)


def _clone(cg, s):
    return cg.Species(s.ux.clone(), s.uy.clone(), s.uz.clone(), s.cell.clone(), s.id.clone())


def _chain(w, want_flag_step1):
    """Steps 0 and 1 as bench.py runs them.  Returns host copies of step 1's
    input (step 0's output), of its binned particles before and after the
    scatter, the offsets, the pair count, and device handles for a re-run."""
    torch = torch_cuda()
    import paper_2206_02937_gb300 as cg
    cg.build()
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    A = [to_species(torch, w.e), to_species(torch, w.g)]
    B = [cg.Species.empty_like(A[0]), cg.Species.empty_like(A[1])]
    p0 = cg.compton_bin_pairs(ctx, A[0], A[1], B[0], B[1], 0)
    cg.compton_scatter_step(ctx, B[0], B[1], p0, cg.MODE_PLAIN, 0, None, None)
    torch.cuda.synchronize()
    inp = [species_np(B[0]), species_np(B[1])]
    p1 = cg.compton_bin_pairs(ctx, B[0], B[1], A[0], A[1], 1)
    torch.cuda.synchronize()
    before = [species_np(A[0]), species_np(A[1])]
    saved = [_clone(cg, A[0]), _clone(cg, A[1])]
    cg.compton_get_stats(ctx, reset=True)
    flag = torch.zeros(max(1, p1.max_pairs), dtype=torch.uint8, device="cuda") if want_flag_step1 else None
    cg.compton_scatter_step(ctx, A[0], A[1], p1, cg.MODE_PLAIN, 1, None, flag)
    torch.cuda.synchronize()
    assert cg.compton_check(ctx) == cg.COMPTON_OK
    stats = cg.compton_get_stats(ctx, reset=True)
    n_pairs = int(stats["pairs_tested"])
    out = dict(ctx=ctx, cg=cg, torch=torch, pairs=p1, saved=saved, inp=inp, before=before,
               after=[species_np(A[0]), species_np(A[1])], n_pairs=n_pairs, stats=stats,
               off_e=_dev_array(torch, p1.off_e_dev, w.n_cells + 1).astype(np.int64),
               off_g=_dev_array(torch, p1.off_g_dev, w.n_cells + 1).astype(np.int64),
               flag=None if flag is None else flag.cpu().numpy()[:n_pairs])
    return out


def _pair_index(off_e, off_g):
    m = np.minimum(np.diff(off_e), np.diff(off_g))
    pair_off = np.concatenate([[0], np.cumsum(m)])
    cell = np.repeat(np.arange(m.shape[0]), m)
    j = np.arange(cell.shape[0]) - pair_off[cell]
    return off_e[cell] + j, off_g[cell] + j, pair_off


# ---------------------------------------------------------------------------
# 256 x 256 cells: the whole chained, filtered step against the oracle's step
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def chain256():
    w = wl.c2(256, 256, 64, seed=2)
    r = _chain(w, want_flag_step1=True)
    r["cg"].compton_destroy(r["ctx"])
    o = oracle.step(w.n_cells, w.w_over_v, w.dt, w.seed, 1, r["inp"][0], r["inp"][1])
    return w, r, o


def test_chained_binning_in_place_matches_oracle(chain256):
    w, r, o = chain256
    for s, inp, perm, off, off_o in ((0, r["inp"][0], o["e_perm"], r["off_e"], o["e_off"]),
                                     (1, r["inp"][1], o["g_perm"], r["off_g"], o["g_off"])):
        assert np.array_equal(off, off_o)
        for key in ("id", "cell") + MOM:
            assert np.array_equal(r["before"][s][key], inp[key][perm]), key
    assert r["n_pairs"] == o["n_pairs"]
    # more scatter tiles than persistent CTAs (152 SMs x 4): every CTA takes
    # several tiles with the candidate filter on
    assert r["n_pairs"] > 4 * 152 * 4 * 1024


def test_chained_filtered_decisions_and_momenta_match_oracle(chain256):
    w, r, o = chain256
    ie, ig, _ = _pair_index(r["off_e"], r["off_g"])
    flag, flag_o = r["flag"].astype(np.int32), o["flag"]
    differ = np.nonzero(flag != flag_o)[0]
    for p in differ:
        assert abs(oracle.bernoulli_u0(w.seed, 1, int(p)) - o["P"][p]) < 1e-6
    assert differ.size <= 3
    ok = np.ones(r["n_pairs"], dtype=bool)
    ok[differ] = False
    ub, kb = _mom(r["before"][0], ie), _mom(r["before"][1], ig)
    ua, ka = _mom(r["after"][0], ie), _mom(r["after"][1], ig)
    uo, ko = o["e_out"][:, ie], o["g_out"][:, ig]
    scale = energy_scale(ub, kb)
    du = np.linalg.norm(ua - uo, axis=0)
    dk = np.linalg.norm(ka - ko, axis=0)
    assert np.all(du[ok] <= 1e-5 * scale[ok])
    assert np.all(dk[ok] <= 1e-5 * scale[ok])
    # pairs that did not collide (and unpaired particles) are untouched
    miss = ok & (flag == 0)
    assert np.array_equal(ua[:, miss], ub[:, miss]) and np.array_equal(ka[:, miss], kb[:, miss])
    paired_e = np.zeros(w.n_e, dtype=bool)
    paired_e[ie] = True
    paired_g = np.zeros(w.n_g, dtype=bool)
    paired_g[ig] = True
    assert np.array_equal(_mom(r["after"][0])[:, ~paired_e], _mom(r["before"][0])[:, ~paired_e])
    assert np.array_equal(_mom(r["after"][1])[:, ~paired_g], _mom(r["before"][1])[:, ~paired_g])
    # every collision of the step took place
    hit = ok & (flag == 1)
    assert hit.sum() > 50000
    assert int(r["stats"]["scatters"]) == int(flag.sum())


# ---------------------------------------------------------------------------
# 512 x 512 cells: the benchmark's call, at its size
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def timed(c2_full):
    w = c2_full
    r = _chain(w, want_flag_step1=False)
    torch, cg = r["torch"], r["cg"]
    try:
        # the same step with every pair's probability and flag requested
        S = r["saved"]
        P = torch.zeros(max(1, r["pairs"].max_pairs), dtype=torch.float32, device="cuda")
        F = torch.zeros(max(1, r["pairs"].max_pairs), dtype=torch.uint8, device="cuda")
        cg.compton_scatter_step(r["ctx"], S[0], S[1], r["pairs"], cg.MODE_PLAIN, 1, P, F)
        torch.cuda.synchronize()
        assert cg.compton_check(r["ctx"]) == cg.COMPTON_OK
        r["full_after"] = [species_np(S[0]), species_np(S[1])]
        r["P"] = P.cpu().numpy()[:r["n_pairs"]]
        r["F"] = F.cpu().numpy()[:r["n_pairs"]]
        del r["saved"]
    finally:
        cg.compton_destroy(r["ctx"])
    return w, r


def test_timed_binning_matches_oracle_sort(timed):
    """Offsets of every cell against a histogram of the input; the order of
    3000 sampled cells (and the first and last) against the oracle's sort of
    those cells' particles."""
    w, r = timed
    rng = np.random.default_rng(5)
    cells = np.unique(np.concatenate([rng.choice(w.n_cells, 3000, replace=False), [0, w.n_cells - 1]]))
    for s, stream, off in ((0, 1, r["off_e"]), (1, 2, r["off_g"])):
        inp = r["inp"][s]
        cnt = np.bincount(inp["cell"], minlength=w.n_cells)
        assert np.array_equal(off, np.concatenate([[0], np.cumsum(cnt)]))
        # step 0's output is in cell order: each sampled cell's input is one run
        assert np.all(np.diff(inp["cell"]) >= 0)
        sel = np.concatenate([np.arange(off[c], off[c + 1]) for c in cells])
        perm, off_o = oracle.sort_species(inp["cell"][sel], inp["id"][sel], w.n_cells, w.seed, 1, stream)
        for key in ("id", "cell") + MOM:
            assert np.array_equal(r["before"][s][key][sel], inp[key][sel][perm]), key
    m = np.minimum(np.diff(r["off_e"]), np.diff(r["off_g"]))
    assert r["n_pairs"] == int(m.sum())


def test_timed_call_equals_full_evaluation(timed):
    w, r = timed
    for s in (0, 1):
        for key in MOM:
            assert np.array_equal(r["after"][s][key], r["full_after"][s][key]), key
    # the particles whose momenta the timed call changed are exactly the
    # flagged pairs of the full evaluation
    ie, ig, _ = _pair_index(r["off_e"], r["off_g"])
    changed = np.zeros(r["n_pairs"], dtype=bool)
    for s, idx in ((0, ie), (1, ig)):
        for key in MOM:
            changed |= r["after"][s][key][idx] != r["before"][s][key][idx]
    assert np.array_equal(changed, r["F"] == 1)


def test_timed_sampled_pairs_match_oracle(timed):
    w, r = timed
    ie, ig, pair_off = _pair_index(r["off_e"], r["off_g"])
    n = r["n_pairs"]
    rng = np.random.default_rng(3)
    first = np.arange(min(2000, n))
    sample = np.unique(np.concatenate([rng.choice(n, 5000, replace=False),
                                       first[r["F"][first] == 1], [0, n - 1]]))
    flips, hits = 0, 0
    for p in sample:
        c = int(np.searchsorted(pair_off, p, side="right") - 1)
        u = _mom(r["before"][0], ie[p])
        k = _mom(r["before"][1], ig[p])
        dens = max(r["off_e"][c + 1] - r["off_e"][c], r["off_g"][c + 1] - r["off_g"][c]) * w.w_over_v
        uo, ko, P, f, _ = oracle.scatter_event(u, k, dens, w.dt, w.seed, 1, int(p))
        assert abs(r["P"][p] - P) <= 2e-5 * P + 1e-9
        if r["F"][p] != f:
            assert abs(oracle.bernoulli_u0(w.seed, 1, int(p)) - P) < 1e-6
            flips += 1
            continue
        hits += f
        scale = energy_scale(u[:, None], k[:, None])[0]
        assert np.linalg.norm(_mom(r["after"][0], ie[p]) - uo) <= 1e-5 * scale
        assert np.linalg.norm(_mom(r["after"][1], ig[p]) - ko) <= 1e-5 * scale
    assert flips <= 3
    assert hits >= 50


def test_chained_per_particle_relative_error(chain256):
    """Momentum error of each collided particle relative to its own oracle
    momentum (not to the pair's energy scale): within 1e-5 for both species.
    Printed as a distribution, split by the FP32 / FP64 gamma eps branch."""
    w, r, o = chain256
    ie, ig, _ = _pair_index(r["off_e"], r["off_g"])
    hit = np.nonzero((r["flag"].astype(np.int32) == 1) & (o["flag"] == 1))[0]
    ua, ka = _mom(r["after"][0], ie[hit]), _mom(r["after"][1], ig[hit])
    uo, ko = o["e_out"][:, ie[hit]], o["g_out"][:, ig[hit]]
    ub, kb = _mom(r["before"][0], ie[hit]), _mom(r["before"][1], ig[hit])
    rel_u = np.linalg.norm(ua - uo, axis=0) / np.linalg.norm(uo, axis=0)
    rel_k = np.linalg.norm(ka - ko, axis=0) / np.linalg.norm(ko, axis=0)
    gamma = np.sqrt(1 + (ub ** 2).sum(0))
    eps = np.linalg.norm(kb, axis=0)
    ge = gamma * eps
    for name, rel in (("electron", rel_u), ("photon", rel_k)):
        q = np.quantile(rel, [0.5, 0.9, 0.99, 0.999, 1.0])
        print(f"\n{name} relative momentum error over {rel.size} collisions: "
              f"median {q[0]:.2e} p90 {q[1]:.2e} p99 {q[2]:.2e} p99.9 {q[3]:.2e} max {q[4]:.2e}")
        for lo, hi in ((0, 8), (8, 1e30)):
            m = (ge >= lo) & (ge < hi)
            if m.any():
                print(f"  gamma*eps in [{lo}, {hi}): {m.sum()} collisions, max {rel[m].max():.2e}, "
                      f"p99 {np.quantile(rel[m], 0.99):.2e}")
        worst = np.argsort(rel)[-3:]
        for i in worst:
            print(f"  worst: rel {rel[i]:.2e} gamma {gamma[i]:.4g} eps {eps[i]:.4g} |u'| "
                  f"{np.linalg.norm(uo[:, i]):.4g} |k'| {np.linalg.norm(ko[:, i]):.4g}")
    assert rel_u.max() <= 1e-5 and rel_k.max() <= 1e-5
