"""Pins of the oracle's unequal-weight step (P_max = 2 sigma_T c dt max w of
Sec. 3.2 per pair; pair density max(N_e, N_g) max(w_e, w_g); weight
rejection of the heavier partner):

  * equal weights reduce it to the unweighted step, bit for bit;
  * the sorted weights follow the particles;
  * the expected number of real events per step, sum of min(w_e, w_g) over
    colliding pairs, equals the rate n_e n_g sigma v dt of the two real
    densities (electrons at rest and photons of energy 1: x = 1, v = 1,
    sigma_KN(1) / sigma_T = 0.43072784191504 from the textbook formula);
  * the heavier partner takes its new momentum in a fraction
    w_light / w_heavy of the collisions, the lighter one always;
  * real energy is conserved on average.
"""
import numpy as np

import oracle
from paper_2206_02937_gb300 import workloads as wl

S_KN_1 = 0.43072784191504


def _beam_cells(n_cells, ne, ng, we, wg):
    """Electrons at rest (weight we), photons of momentum (0, 0, 1) (weight wg)."""
    e = dict(ux=np.zeros(n_cells * ne, np.float32), uy=np.zeros(n_cells * ne, np.float32),
             uz=np.zeros(n_cells * ne, np.float32), cell=np.repeat(np.arange(n_cells), ne).astype(np.int32),
             id=np.arange(n_cells * ne, dtype=np.uint32), w=np.full(n_cells * ne, we, np.float32))
    g = dict(ux=np.zeros(n_cells * ng, np.float32), uy=np.zeros(n_cells * ng, np.float32),
             uz=np.ones(n_cells * ng, np.float32), cell=np.repeat(np.arange(n_cells), ng).astype(np.int32),
             id=np.arange(n_cells * ng, dtype=np.uint32), w=np.full(n_cells * ng, wg, np.float32))
    return e, g


def test_equal_weights_reduce_to_the_unweighted_step():
    w = wl.c1()
    ref = oracle.step(w.n_cells, w.w_over_v, w.dt, w.seed, 0, w.e, w.g)
    e = dict(w.e, w=np.full(w.n_e, w.w_over_v, np.float32))
    g = dict(w.g, w=np.full(w.n_g, w.w_over_v, np.float32))
    for ee, gg in ((e, g), (w.e, w.g), (e, w.g)):
        out = oracle.step_weighted(w.n_cells, w.w_over_v, w.dt, w.seed, 0, ee, gg)
        assert np.array_equal(out["P"], ref["P"]) and np.array_equal(out["flag"], ref["flag"])
        assert np.array_equal(out["e_out"], ref["e_out"]) and np.array_equal(out["g_out"], ref["g_out"])
        assert np.array_equal(out["upd"], 3 * ref["flag"])
    assert ref["flag"].sum() > 50


def test_sorted_weights_follow_the_particles():
    w = wl.c1()
    rng = np.random.default_rng(5)
    e = dict(w.e, w=rng.uniform(0.5, 2.0, w.n_e).astype(np.float32))
    g = dict(w.g, w=rng.uniform(0.5, 2.0, w.n_g).astype(np.float32))
    out = oracle.step_weighted(w.n_cells, w.w_over_v, w.dt, w.seed, 3, e, g)
    assert np.array_equal(out["e_w"], e["w"][out["e_perm"]].astype(np.float64))
    assert np.array_equal(out["g_w"], g["w"][out["g_perm"]].astype(np.float64))


def _collisions(we, wg, ne=40, ng=100, n_cells=400, steps=100, dt=0.01):
    e, g = _beam_cells(n_cells, ne, ng, we, wg)
    real, n_coll, upd_e, upd_g, d_energy = 0.0, 0, 0, 0, []
    for st in range(steps):
        out = oracle.step_weighted(n_cells, 1.0, dt, 77, st, e, g)
        f = out["flag"].astype(bool)
        n_coll += int(f.sum())
        real += f.sum() * min(we, wg)
        upd_e += int((out["upd"][f] & 1).sum())
        upd_g += int(((out["upd"][f] >> 1) & 1).sum())
        gam = np.sqrt(1.0 + (out["e_out"] ** 2).sum(0))
        eps = np.sqrt((out["g_out"] ** 2).sum(0))
        d_energy.append(we * (gam - 1.0).sum() + wg * (eps - 1.0).sum())
    return real / steps, n_coll, upd_e, upd_g, np.array(d_energy)


def test_real_event_rate_and_weight_rejection():
    ne, ng, n_cells, dt = 40, 100, 400, 0.01
    for we, wg in ((0.01, 0.002), (0.002, 0.01)):
        rate, n_coll, upd_e, upd_g, d_energy = _collisions(we, wg, ne, ng, n_cells, dt=dt)
        # real events per step: n_e n_g sigma v dt V (V = 1 per cell), linear
        # regime (1 - exp(-a) = a (1 - a/2), a < 0.005)
        expect = n_cells * (ne * we) * (ng * wg) * S_KN_1 * 1.0 * dt
        sig = expect / np.sqrt(n_coll)
        assert abs(rate - expect) < 5.0 * sig + 0.005 * expect, (rate, expect)
        # weight rejection: the heavier partner updates in w_light / w_heavy
        heavy, light = (upd_e, upd_g) if we > wg else (upd_g, upd_e)
        ratio = min(we, wg) / max(we, wg)
        assert light == n_coll
        sd = np.sqrt(ratio * (1.0 - ratio) / n_coll)
        assert abs(heavy / n_coll - ratio) < 5.0 * sd
        # real energy change per step: zero mean (t statistic), while a
        # heavier partner updated every time would move it by
        # (w_heavy - w_light) per unit transferred
        t = d_energy.mean() / (d_energy.std(ddof=1) / np.sqrt(d_energy.size))
        assert abs(t) < 5.0, t
        assert d_energy.std() > 0.0
