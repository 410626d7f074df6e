"""Pins of the oracle's No-Time-Counter step (Sec. 3.1, second step; Bird
1989): candidate counts are unbiased, the collision rate equals the pairing
method's in the linear regime, every cell conserves energy and momentum, a
single pair can collide several times in one step, and empty species give
no candidates."""
import numpy as np

import oracle
from paper_2206_02937_gb300 import workloads as wl


def _energy_momentum(o, w):
    ue, kg = o["e_out"], o["g_out"]
    ce = np.repeat(np.arange(w.n_cells), np.diff(o["e_off"]))
    cg = np.repeat(np.arange(w.n_cells), np.diff(o["g_off"]))
    E = np.zeros(w.n_cells)
    p = np.zeros((3, w.n_cells))
    np.add.at(E, ce, np.sqrt(1.0 + (ue ** 2).sum(0)))
    np.add.at(E, cg, np.sqrt((kg ** 2).sum(0)))
    for i in range(3):
        np.add.at(p[i], ce, ue[i])
        np.add.at(p[i], cg, kg[i])
    return E, p


def test_candidate_counts_unbiased_and_rate_matches_pairing():
    w = wl.c2(24, 24, 64, seed=4)
    o = oracle.ntc_step(w.n_cells, w.w_over_v, w.dt, w.seed, 2, w.e, w.g)
    ne, ng = np.diff(o["e_off"]), np.diff(o["g_off"])
    expect = ne * ng * w.w_over_v * 2.0 * w.dt
    # floor(E + U): every cell within one of its expectation, the sum unbiased
    assert np.all(np.abs(o["n_cand"] - expect) < 1.0)
    assert abs(o["n_cand"].sum() - expect.sum()) < 4.0 * np.sqrt(w.n_cells / 12.0)
    # NTC and random pairing estimate the same collision count (linear regime)
    rates = []
    for st in range(4):
        a = oracle.ntc_step(w.n_cells, w.w_over_v, w.dt, w.seed, 10 + st, w.e, w.g)["n_coll"].sum()
        b = oracle.step(w.n_cells, w.w_over_v, w.dt, w.seed, 10 + st, w.e, w.g)["flag"].sum()
        rates.append((a, b))
    a, b = np.array(rates).sum(0)
    assert abs(a / b - 1.0) < 4.0 * np.sqrt(1.0 / a + 1.0 / b) + 0.03, (a, b)


def test_every_cell_conserves_energy_and_momentum():
    w = wl.c2(12, 12, 48, seed=5)
    before = oracle.ntc_step(w.n_cells, w.w_over_v, 0.0, w.seed, 3, w.e, w.g)  # dt = 0: no candidates
    assert before["total_candidates"] == 0
    o = oracle.ntc_step(w.n_cells, w.w_over_v, w.dt, w.seed, 3, w.e, w.g)
    assert o["n_coll"].sum() > 100
    E0, p0 = _energy_momentum(before, w)
    E1, p1 = _energy_momentum(o, w)
    assert np.all(np.abs(E1 - E0) <= 1e-12 * E0)
    assert np.all(np.linalg.norm(p1 - p0, axis=0) <= 1e-12 * E0)


def test_single_pair_collides_repeatedly():
    # one electron and one photon with a large candidate count: the same pair
    # is drawn again and again and collides in sequence
    rng = wl.rng_for(6)
    e = wl._species(3.0 * wl.isotropic(rng, 1), np.zeros(1, dtype=np.int64))
    g = wl._species(0.3 * wl.isotropic(rng, 1), np.zeros(1, dtype=np.int64))
    w = wl.Workload("one pair", 1, 200.0, 0.05, 11, 1, e, g)  # E = 1 * 1 * 200 * 2 * 0.05 = 20
    o = oracle.ntc_step(1, 200.0, 0.05, 11, 0, e, g)
    assert o["n_cand"][0] in (20, 21)
    assert o["n_coll"][0] >= 2
    E0, p0 = _energy_momentum(oracle.ntc_step(1, 200.0, 0.0, 11, 0, e, g), w)
    E1, p1 = _energy_momentum(o, w)
    assert abs(E1[0] - E0[0]) <= 1e-12 * E0[0]
    assert np.linalg.norm(p1[:, 0] - p0[:, 0]) <= 1e-12 * E0[0]


def test_one_sided_cells_have_no_candidates():
    rng = wl.rng_for(7)
    e = wl._species(wl.isotropic(rng, 40), np.arange(40) % 4)
    g = wl._species(0.1 * wl.isotropic(rng, 30), 4 + np.arange(30) % 3)
    o = oracle.ntc_step(8, 1.0, 0.05, 1, 0, e, g)
    assert o["total_candidates"] == 0 and o["n_coll"].sum() == 0
    assert np.allclose(o["e_out"], np.stack([e["ux"], e["uy"], e["uz"]])[:, o["e_perm"]])
