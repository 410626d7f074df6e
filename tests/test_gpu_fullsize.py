"""Parity at the benchmark's full size (2D 512 x 512 cells, ~16.8M pairs per
step, the launch configuration bench.py times), on sampled outputs the oracle
recomputes one by one, and on properties that hold at any size."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import energy_scale, gpu_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full(c2_full):
    return c2_full, gpu_step(c2_full, step=3)


def test_full_size_binning_properties(full):
    w, g = full
    C = w.n_cells
    ce = np.bincount(w.e["cell"], minlength=C)
    cg = np.bincount(w.g["cell"], minlength=C)
    assert np.array_equal(np.diff(g["off_e"].astype(np.int64)), ce)
    assert np.array_equal(np.diff(g["off_g"].astype(np.int64)), cg)
    assert np.all(np.diff(g["before_e"]["cell"]) >= 0)
    assert np.all(np.diff(g["before_g"]["cell"]) >= 0)
    # the sorted output is a permutation of the input (ids)
    assert np.array_equal(np.sort(g["before_e"]["id"]), np.sort(w.e["id"]))
    assert g["n_pairs"] == int(np.minimum(ce, cg).sum())
    # sampled cells: order by (key, id) from the oracle's Philox
    rng = np.random.default_rng(0)
    for c in rng.choice(C, 60, replace=False):
        for s, off, stream in (("before_e", g["off_e"], 1), ("before_g", g["off_g"], 2)):
            ids = g[s]["id"][off[c]:off[c + 1]]
            keys = [(oracle.pair_key(w.seed, 3, stream, int(i)), int(i)) for i in ids]
            assert keys == sorted(keys)


def test_full_size_sampled_pairs_match_oracle(full):
    w, g = full
    C = w.n_cells
    off_e, off_g = g["off_e"].astype(np.int64), g["off_g"].astype(np.int64)
    m = np.minimum(np.diff(off_e), np.diff(off_g))
    pair_off = np.concatenate([[0], np.cumsum(m)])
    rng = np.random.default_rng(1)
    sample = np.concatenate([rng.choice(g["n_pairs"], 3000, replace=False),
                             np.nonzero(g["flag"])[0][:1000], [0, g["n_pairs"] - 1]])
    flips = 0
    for p in sample:
        c = int(np.searchsorted(pair_off, p, side="right") - 1)
        j = p - pair_off[c]
        ie, ig = off_e[c] + j, off_g[c] + j
        u = np.array([g["before_e"][a][ie] for a in ("ux", "uy", "uz")], dtype=np.float64)
        k = np.array([g["before_g"][a][ig] for a in ("ux", "uy", "uz")], dtype=np.float64)
        n_dens = max(off_e[c + 1] - off_e[c], off_g[c + 1] - off_g[c]) * w.w_over_v
        uo, ko, P, f, _ = oracle.scatter_event(u, k, n_dens, w.dt, w.seed, 3, int(p))
        assert abs(g["P"][p] - P) <= 2e-5 * P + 1e-9
        u0 = oracle.bernoulli_u0(w.seed, 3, int(p))
        if g["flag"][p] != f:
            assert abs(u0 - P) < 1e-6
            flips += 1
            continue
        scale = energy_scale(u[:, None], k[:, None])[0]
        ua = np.array([g["after_e"][a][ie] for a in ("ux", "uy", "uz")], dtype=np.float64)
        ka = np.array([g["after_g"][a][ig] for a in ("ux", "uy", "uz")], dtype=np.float64)
        assert np.linalg.norm(ua - uo) <= 1e-5 * scale
        assert np.linalg.norm(ka - ko) <= 1e-5 * scale
    assert flips <= 3


def test_full_size_conservation_and_rate(full):
    w, g = full
    off_e, off_g = g["off_e"].astype(np.int64), g["off_g"].astype(np.int64)
    m = np.minimum(np.diff(off_e), np.diff(off_g))
    cell = np.repeat(np.arange(w.n_cells), m)
    j = np.arange(cell.shape[0]) - np.concatenate([[0], np.cumsum(m)])[cell]
    ie, ig = off_e[cell] + j, off_g[cell] + j
    hit = np.nonzero(g["flag"])[0]
    assert g["stats"]["scatters"] == hit.size
    mom = lambda s, idx: np.stack([s[a][idx] for a in ("ux", "uy", "uz")]).astype(np.float64)  # noqa: E731
    ub, kb = mom(g["before_e"], ie[hit]), mom(g["before_g"], ig[hit])
    ua, ka = mom(g["after_e"], ie[hit]), mom(g["after_g"], ig[hit])
    Eb, Ea = energy_scale(ub, kb), energy_scale(ua, ka)
    assert np.all(np.abs(Ea - Eb) <= 2e-6 * Eb)
    assert np.all(np.linalg.norm(ua + ka - ub - kb, axis=0) <= 2e-6 * Eb)
    # the count of collisions agrees with the sum of probabilities
    Psum = float(g["P"].astype(np.float64).sum())
    var = float((g["P"] * (1 - g["P"])).astype(np.float64).sum())
    assert abs(hit.size - Psum) < 6 * np.sqrt(var)
