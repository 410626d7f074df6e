"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: a
high-precision evaluation of the textbook closed form (mpmath, 50 digits),
quadrature of the differential cross section (scipy), exact rational series
(sympy), limits with a closed form (Thomson, head-on, dipole), conservation
laws, brute force on tiny inputs, or a chi-square against the analytic
distribution.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 50


def kn_mp(x):
    """Textbook Klein-Nishina total cross section / sigma_T, 50 digits."""
    x = mpmath.mpf(x)
    L = mpmath.log(1 + 2 * x)
    return mpmath.mpf(3) / 4 * ((1 + x) / x**3 * (2 * x * (1 + x) / (1 + 2 * x) - L)
                                + L / (2 * x) - (1 + 3 * x) / (1 + 2 * x) ** 2)


# --------------------------------------------------------------------------
# Klein-Nishina total cross section (Sec. 3.2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("x", [1e-9, 1e-6, 1e-4, 1e-3, 1e-2, 0.1, 0.2, 0.2499999, 0.25, 0.3,
                               0.5, 1.0, 3.0, 10.0, 100.0, 1e4, 1e6])
def test_kn_sigma_matches_50_digit_closed_form(x):
    ref = float(kn_mp(x))
    assert abs(oracle.kn_sigma(x) - ref) <= 2e-14 * ref


def test_kn_sigma_published_style_values():
    # values of the closed form at 50 digits, rounded to 14 significant digits
    for x, ref in [(1e-4, 0.99980005198670), (1e-2, 0.98050701926190),
                   (1.0, 0.43072784191504), (100.0, 0.021510621648694)]:
        assert oracle.kn_sigma(x) == pytest.approx(ref, rel=1e-13)


def test_thomson_limit():
    # s(x) -> 1 - 2x as x -> 0 (Thomson limit, first-order recoil)
    for x in (1e-12, 1e-10, 1e-8):
        assert abs(oracle.kn_sigma(x) - (1 - 2 * x)) < 1e-15
    assert oracle.kn_sigma(0.0) == 1.0


def test_high_energy_asymptote():
    # s(x) ~ 3/(8x) (ln 2x + 1/2) for x >> 1
    x = 1e6
    asym = 3.0 / (8 * x) * (math.log(2 * x) + 0.5)
    assert oracle.kn_sigma(x) == pytest.approx(asym, rel=3e-6)


def test_series_coefficients_match_sympy():
    sympy = pytest.importorskip("sympy")
    X = sympy.symbols("x", positive=True)
    L = sympy.log(1 + 2 * X)
    s = sympy.Rational(3, 4) * ((1 + X) / X**3 * (2 * X * (1 + X) / (1 + 2 * X) - L)
                                + L / (2 * X) - (1 + 3 * X) / (1 + 2 * X) ** 2)
    ser = sympy.series(s, X, 0, 9).removeO()
    for n in range(9):
        exact = ser.coeff(X, n)
        assert oracle.kn_series_coef(n) == pytest.approx(float(exact), rel=1e-15, abs=1e-300)
    # the first terms quoted for the Thomson series: 1 - 2x + 26/5 x^2 - 133/10 x^3
    assert [oracle.kn_series_coef(i) for i in range(4)] == pytest.approx([1, -2, 5.2, -13.3], rel=1e-15)


def test_kn_monotone_decreasing():
    xs = np.logspace(-6, 6, 400)
    s = np.array([oracle.kn_sigma(x) for x in xs])
    assert np.all(np.diff(s) < 0)
    assert np.all((s > 0) & (s <= 1))


# --------------------------------------------------------------------------
# Differential cross section and its cumulative (sampling of Sec. 3.1 step 3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("x", [1e-4, 1e-2, 0.3, 1.0, 100.0, 1e4])
def test_differential_integrates_to_total(x):
    from scipy.integrate import quad
    val, err = quad(lambda t: oracle.kn_dsigma_dt(x, t), 0.0, 2.0, epsabs=0, epsrel=1e-13,
                    limit=400, points=[1.0 / x] if x > 1 else None)
    assert val == pytest.approx(kn_mp(x), rel=1e-11)


def test_differential_matches_klein_nishina_angular_formula():
    # dsigma/dOmega = r_e^2/2 (e1/e)^2 (e1/e + e/e1 - sin^2), sigma_T = 8 pi r_e^2 / 3
    for x in (0.01, 1.0, 50.0):
        for mu in (-0.9, 0.0, 0.5, 0.99):
            ratio = 1.0 / (1.0 + x * (1 - mu))
            dsdo = 0.5 * ratio**2 * (ratio + 1 / ratio - (1 - mu**2))
            per_t = 2 * math.pi * dsdo / (8 * math.pi / 3)
            assert oracle.kn_dsigma_dt(x, 1 - mu) == pytest.approx(per_t, rel=1e-14)


@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.1, 0.24, 0.26, 0.3, 1.0, 7.0, 100.0, 5e3])
@pytest.mark.parametrize("t", [1e-6, 0.01, 0.4, 0.5 / 0.26, 1.0, 1.7, 2.0])
def test_cdf_matches_quadrature(x, t):
    from scipy.integrate import quad
    ref, _ = quad(lambda tt: oracle.kn_dsigma_dt(x, tt), 0.0, t, epsabs=0, epsrel=1e-13, limit=400)
    assert oracle.kn_cdf(x, t) == pytest.approx(ref, rel=2e-12)


def test_cdf_branch_boundary_continuous():
    # series branch (x t < 1/2) and closed branch meet without a jump
    for x in (0.25, 0.26, 0.4, 1.0):
        t = 0.5 / x
        lo = oracle.kn_cdf(x, t * (1 - 1e-12))
        hi = oracle.kn_cdf(x, t * (1 + 1e-12))
        assert abs(hi - lo) < 1e-11 * abs(lo)


@pytest.mark.parametrize("x", [1e-5, 1e-3, 0.2, 1.0, 30.0, 2000.0])
def test_cdf_at_two_is_total(x):
    assert oracle.kn_cdf(x, 2.0) == pytest.approx(float(kn_mp(x)), rel=1e-12)


def test_sample_inverts_cdf():
    rng = np.random.default_rng(7)
    for x in (1e-5, 0.01, 0.7, 15.0, 900.0):
        tot = oracle.kn_cdf(x, 2.0)
        for u in rng.uniform(0, 1, 20):
            t = oracle.kn_sample_t(x, u)
            assert 0.0 <= t <= 2.0
            assert oracle.kn_cdf(x, t) == pytest.approx(u * tot, rel=1e-13, abs=1e-16)


def _chi2_pvalue(counts, expected):
    from scipy.stats import chi2
    stat = float(np.sum((counts - expected) ** 2 / expected))
    return chi2.sf(stat, len(counts) - 1)


@pytest.mark.parametrize("x", [1e-4, 1e-2, 1.0, 100.0])
def test_sampled_angles_chi_square(x):
    # 2e4 inverse-CDF draws on a uniform u grid with random offsets, 40 bins
    # in t; expected counts from the analytic differential by quadrature.
    from scipy.integrate import quad
    rng = np.random.default_rng(11)
    us = rng.uniform(0, 1, 20000)
    ts = np.array([oracle.kn_sample_t(x, u) for u in us])
    edges = np.linspace(0, 2, 41)
    counts, _ = np.histogram(ts, edges)
    tot = float(kn_mp(x))
    probs = np.array([quad(lambda t: oracle.kn_dsigma_dt(x, t), a, b, epsrel=1e-12)[0]
                      for a, b in zip(edges[:-1], edges[1:])]) / tot
    assert _chi2_pvalue(counts, probs * len(ts)) > 1e-3


def test_dipole_limit():
    # x -> 0: the angular distribution of Thomson scattering, (1 + cos^2) dmu
    rng = np.random.default_rng(3)
    us = rng.uniform(0, 1, 20000)
    mu = np.array([1 - oracle.kn_sample_t(1e-9, u) for u in us])
    edges = np.linspace(-1, 1, 21)
    counts, _ = np.histogram(mu, edges)
    F = lambda m: (m + m**3 / 3)  # noqa: E731  antiderivative of 1 + mu^2
    probs = (F(edges[1:]) - F(edges[:-1])) / (F(1) - F(-1))
    assert _chi2_pvalue(counts, probs * len(mu)) > 1e-3


def test_scattered_energy_ratio_chi_square():
    # energy ratio e1'/e' = 1/(1 + x t): its histogram follows from the same
    # analytic cumulative through the monotone map t -> ratio
    x = 1.0
    rng = np.random.default_rng(5)
    us = rng.uniform(0, 1, 20000)
    ratio = np.array([1.0 / (1.0 + x * oracle.kn_sample_t(x, u)) for u in us])
    r_edges = np.linspace(1.0 / (1 + 2 * x), 1.0, 31)
    counts, _ = np.histogram(ratio, r_edges)
    t_edges = (1.0 / r_edges - 1.0) / x  # decreasing
    tot = float(kn_mp(x))
    from scipy.integrate import quad
    probs = np.array([quad(lambda t: oracle.kn_dsigma_dt(x, t), t_edges[i + 1], t_edges[i],
                           epsrel=1e-12)[0] for i in range(30)]) / tot
    assert _chi2_pvalue(counts, probs * len(ratio)) > 1e-3


# --------------------------------------------------------------------------
# Invariants and boosts (Sec. 3.2: boost to the lepton frame and back)
# --------------------------------------------------------------------------
def _x_v_mp(u, k):
    u = [mpmath.mpf(float(c)) for c in u]
    k = [mpmath.mpf(float(c)) for c in k]
    uu = sum(c * c for c in u)
    g = mpmath.sqrt(1 + uu)
    e = mpmath.sqrt(sum(c * c for c in k))
    uk = sum(a * b for a, b in zip(u, k))
    x = g * e - uk
    v = x / (g * e)
    return float(x), float(v)


def _rand_dir(rng):
    z = rng.uniform(-1, 1)
    ph = rng.uniform(0, 2 * np.pi)
    s = math.sqrt(1 - z * z)
    return np.array([s * math.cos(ph), s * math.sin(ph), z])


def test_invariants_match_high_precision():
    rng = np.random.default_rng(1)
    for _ in range(300):
        g = 10 ** rng.uniform(0, 5)
        e = 10 ** rng.uniform(-6, 1)
        u = np.float32(math.sqrt(g * g - 1) * _rand_dir(rng)).astype(np.float64)
        k = np.float32(e * _rand_dir(rng)).astype(np.float64)
        x, v = oracle.invariants(u, k)
        xr, vr = _x_v_mp(u, k)
        assert x == pytest.approx(xr, rel=1e-13)
        assert v == pytest.approx(vr, rel=1e-13)


def test_invariants_nearly_collinear_high_gamma():
    # co-moving photon at gamma = 1e4, tiny angles: the cancellation-prone case
    for ang in (0.0, 1e-7, 1e-5, 1e-3):
        u = np.array([1e4, 0.0, 0.0], dtype=np.float32).astype(np.float64)
        k = np.array([1e-2 * math.cos(ang), 1e-2 * math.sin(ang), 0.0], dtype=np.float32).astype(np.float64)
        x, v = oracle.invariants(u, k)
        xr, vr = _x_v_mp(u, k)
        assert x == pytest.approx(xr, rel=1e-12)
        assert v == pytest.approx(vr, rel=1e-12)


def test_head_on_and_comoving_limits():
    g = 50.0
    un = math.sqrt(g * g - 1)
    beta = un / g
    e = 0.3
    x, v = oracle.invariants([un, 0, 0], [-e, 0, 0])
    assert x == pytest.approx(g * e * (1 + beta), rel=1e-15)
    assert v == pytest.approx(1 + beta, rel=1e-15)
    x, v = oracle.invariants([un, 0, 0], [e, 0, 0])
    assert x == pytest.approx(e * g * (1 - beta), rel=1e-13)
    assert x == pytest.approx(e / (2 * g), rel=1e-3)
    # electron at rest: x = eps, v = 1
    x, v = oracle.invariants([0, 0, 0], [0.1, 0.2, 0.3])
    assert v == 1.0 and x == pytest.approx(math.sqrt(0.14), rel=1e-15)


def test_boost_gives_rest_frame_energy_and_round_trips():
    rng = np.random.default_rng(2)
    for _ in range(200):
        g = 10 ** rng.uniform(0, 3)
        u = math.sqrt(g * g - 1) * _rand_dir(rng)
        k = 10 ** rng.uniform(-4, 0) * _rand_dir(rng)
        er, kr = oracle.boost_to_rest(u, k)
        x, _ = oracle.invariants(u, k)
        assert er == pytest.approx(x, rel=1e-9)
        assert np.linalg.norm(kr) == pytest.approx(er, rel=1e-9)  # still on shell
        e2, k2 = oracle.boost_to_lab(u, er, kr)
        assert e2 == pytest.approx(np.linalg.norm(k), rel=1e-9)
        assert np.allclose(k2, k, rtol=1e-9, atol=1e-14 * g * g)


def test_boost_matches_explicit_lorentz_matrix():
    # the standard boost matrix with beta = u/gamma, applied to (eps, k)
    rng = np.random.default_rng(9)
    for _ in range(50):
        g = 10 ** rng.uniform(0, 2)
        u = math.sqrt(g * g - 1) * _rand_dir(rng)
        k = 0.1 * _rand_dir(rng)
        b = u / g
        b2 = b @ b
        Lam = np.eye(4)
        Lam[0, 0] = g
        Lam[0, 1:] = Lam[1:, 0] = -g * b
        Lam[1:, 1:] += (g - 1) * np.outer(b, b) / b2
        four = Lam @ np.concatenate([[np.linalg.norm(k)], k])
        er, kr = oracle.boost_to_rest(u, k)
        assert er == pytest.approx(four[0], rel=1e-12)
        assert np.allclose(kr, four[1:], rtol=1e-11, atol=1e-13)


def test_onb_is_orthonormal():
    rng = np.random.default_rng(4)
    dirs = [_rand_dir(rng) for _ in range(200)] + [np.array([0, 0, 1.0]), np.array([0, 0, -1.0]),
                                                  np.array([1.0, 0, 0])]
    for n in dirs:
        b1, b2 = oracle.onb(n)
        M = np.stack([b1, b2, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-14)
        assert np.dot(np.cross(b1, b2), n) == pytest.approx(1.0, abs=1e-14)  # right-handed


# --------------------------------------------------------------------------
# Probability, Bernoulli trial and conservation (Sec. 3.1, Sec. 3.2)
# --------------------------------------------------------------------------
def test_probability_closed_form_and_bernoulli():
    rng = np.random.default_rng(6)
    for i in range(300):
        g = 10 ** rng.uniform(0, 3)
        u = np.float32(math.sqrt(g * g - 1) * _rand_dir(rng)).astype(np.float64)
        k = np.float32(10 ** rng.uniform(-4, 0) * _rand_dir(rng)).astype(np.float64)
        n, dt = 10 ** rng.uniform(-1, 1.5), 0.05
        uo, ko, P, flag, x = oracle.scatter_event(u, k, n, dt, 17, 3, i)
        xr, vr = _x_v_mp(u, k)
        a = n * dt * kn_mp(xr) * vr
        assert P == pytest.approx(float(1 - mpmath.exp(-a)), rel=1e-12)
        # Bernoulli: word i mod 4 of Philox(counter=(i / 4, step, 3, 0), key=(seed, 0))
        r = oracle.philox4x32_10([i >> 2, 3, 3, 0], [17, 0])
        u0 = (int(r[i & 3]) >> 8) / 2.0**24
        assert oracle.bernoulli_u0(17, 3, i) == u0
        assert flag == int(u0 < P)
        if not flag:
            assert np.array_equal(uo, u) and np.array_equal(ko, k)


def test_small_probability_is_linear():
    u, k = [3.0, 0, 0], [0, 1e-3, 0]
    _, _, P, _, x = oracle.scatter_event(u, k, 1e-6, 0.05, 1, 0, 0)
    _, v = oracle.invariants(u, k)
    assert P == pytest.approx(1e-6 * 0.05 * oracle.kn_sigma(x) * v, rel=1e-7)


def _conservation(u, k, uo, ko):
    g0 = math.sqrt(1 + u @ u)
    g1 = math.sqrt(1 + uo @ uo)
    E0 = g0 + np.linalg.norm(k)
    E1 = g1 + np.linalg.norm(ko)
    p0, p1 = u + k, uo + ko
    s0 = E0 * E0 - p0 @ p0
    s1 = E1 * E1 - p1 @ p1
    return abs(E1 - E0) / E0, np.linalg.norm(p1 - p0) / E0, abs(s1 - s0) / (E0 * E0)


def test_scattered_events_conserve_energy_momentum():
    rng = np.random.default_rng(8)
    seen = 0
    for i in range(4000):
        g = 10 ** rng.uniform(0, 3)
        u = math.sqrt(g * g - 1) * _rand_dir(rng)
        k = 10 ** rng.uniform(-4, 0) * _rand_dir(rng)
        uo, ko, P, flag, x = oracle.scatter_event(u, k, 200.0, 0.05, 23, 0, i)
        if not flag:
            continue
        seen += 1
        dE, dp, ds = _conservation(u, k, uo, ko)
        assert dE < 1e-12 and dp < 1e-12 and ds < 1e-11
        # scattered photon energy follows the Compton formula in the rest frame
        er1, _ = oracle.boost_to_rest(u, ko)
        r = oracle.philox4x32_10([i, 0, 4, 0], [23, 0])  # angle draws: stream 4
        t = oracle.kn_sample_t(x, ((int(r[0]) >> 8) + 0.5) / 2.0**24)
        assert er1 == pytest.approx(x / (1 + x * t), rel=1e-8)
    assert seen > 1000


# --------------------------------------------------------------------------
# Binning and pairing (Sec. 3.1 first step), brute force
# --------------------------------------------------------------------------
def test_sort_species_brute_force():
    rng = np.random.default_rng(12)
    n, C = 500, 13
    cell = rng.integers(0, C, n).astype(np.int32)
    pid = rng.permutation(10 * n)[:n].astype(np.uint32)
    perm, off = oracle.sort_species(cell, pid, C, seed=5, step=9, stream=1)
    keyed = sorted(range(n), key=lambda i: (cell[i], oracle.pair_key(5, 9, 1, pid[i]), pid[i]))
    assert list(perm) == keyed
    counts = np.bincount(cell, minlength=C)
    assert list(off) == [0] + list(np.cumsum(counts))


def test_step_pairs_ranks_and_counts():
    rng = np.random.default_rng(13)
    C = 6
    ne, ng = 40, 30
    e = dict(ux=rng.normal(size=ne).astype(np.float32), uy=rng.normal(size=ne).astype(np.float32),
             uz=rng.normal(size=ne).astype(np.float32), cell=rng.integers(0, C, ne).astype(np.int32),
             id=np.arange(ne, dtype=np.uint32))
    g = dict(ux=rng.normal(size=ng).astype(np.float32) * 0.01, uy=rng.normal(size=ng).astype(np.float32) * 0.01,
             uz=rng.normal(size=ng).astype(np.float32) * 0.01, cell=rng.integers(0, C, ng).astype(np.int32),
             id=np.arange(ng, dtype=np.uint32))
    out = oracle.step(C, 0.5, 0.05, 3, 1, e, g)
    ce = np.bincount(e["cell"], minlength=C)
    cg = np.bincount(g["cell"], minlength=C)
    assert out["n_pairs"] == int(np.minimum(ce, cg).sum())
    # every pair evaluated with density max(N_e, N_g) * w/V
    q = 0
    for c in range(C):
        m = min(ce[c], cg[c])
        for j in range(m):
            ie = out["e_perm"][out["e_off"][c] + j]
            ig = out["g_perm"][out["g_off"][c] + j]
            u = np.array([e["ux"][ie], e["uy"][ie], e["uz"][ie]], dtype=np.float64)
            k = np.array([g["ux"][ig], g["uy"][ig], g["uz"][ig]], dtype=np.float64)
            _, _, P, f, _ = oracle.scatter_event(u, k, max(ce[c], cg[c]) * 0.5, 0.05, 3, 1, q)
            assert P == out["P"][q] and f == out["flag"][q]
            q += 1
    # unpaired particles unchanged
    for c in range(C):
        for j in range(min(ce[c], cg[c]), ce[c]):
            ie = out["e_perm"][out["e_off"][c] + j]
            assert out["e_out"][0, out["e_off"][c] + j] == e["ux"][ie]


def test_mean_scatter_count_matches_sum_of_probabilities():
    # the Bernoulli decisions are unbiased: sum(flag) ~ Poisson-binomial(sum P)
    rng = np.random.default_rng(14)
    n = 20000
    u = (3.0 * rng.normal(size=(3, n))).astype(np.float32)
    k = (0.1 * rng.normal(size=(3, n))).astype(np.float32)
    nd = np.full(n, 5.0, dtype=np.float32)
    _, _, P, flag = oracle.pairs(u, k, nd, 0.05, 77, 0)
    mean, var = P.sum(), (P * (1 - P)).sum()
    assert abs(flag.sum() - mean) < 5 * math.sqrt(var)
