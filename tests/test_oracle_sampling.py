"""Distribution pins of the oracle's scattering samplers (no GPU).

u_par (Sec. 3.2.3) against the exact pdf of Eq. uparf by per-bin quadrature,
normalised with scipy's Faddeeva H (chi-square); the phase-function inversion
(Eq. phaseW) against quadrature of W; core-skipping's truncated Gaussian
(Sec. 3.2.4) against its closed-form tail; the recoil shift (Eq. x_f)."""
import numpy as np
import pytest
from scipy import integrate, stats
from scipy.special import wofz


def _bin_mass(x, a, lo, hi):
    # int_lo^hi exp(-u^2)/(a^2+(x-u)^2) du with u = x + a tan(t)
    t0, t1 = np.arctan((lo - x) / a), np.arctan((hi - x) / a)
    f = lambda t: np.exp(-(x + a * np.tan(t)) ** 2) / a
    pts = [p for p in (np.arctan((-x) / a), 0.0) if t0 < p < t1]
    v, _ = integrate.quad(f, t0, t1, points=pts or None, limit=400, epsabs=0, epsrel=1e-10)
    return v


def _chi2_upar(x, a, samples):
    total = np.pi * wofz(abs(x) + 1j * a).real / a      # int exp(-u^2)/(a^2+(x-u)^2) du
    edges = set(np.linspace(-4.5, 4.5 + abs(x), 37))
    for t in np.linspace(-1.45, 1.45, 21):
        e = x + a * np.tan(t)
        if -4.5 < e < 4.5 + abs(x):
            edges.add(e)
    edges = np.array(sorted(edges))
    edges = edges[np.concatenate([[True], np.diff(edges) > 1e-9])]
    mass = np.array([_bin_mass(x, a, edges[i], edges[i + 1]) for i in range(len(edges) - 1)]) / total
    full = np.concatenate([[_bin_mass(x, a, -60.0, edges[0]) / total], mass,
                           [_bin_mass(x, a, edges[-1], 60.0 + abs(x)) / total]])
    counts = np.histogram(samples, bins=np.concatenate([[-np.inf], edges, [np.inf]]))[0]
    n = len(samples)
    exp = full * n
    # merge sparse cells
    obs_m, exp_m, ao, ae = [], [], 0.0, 0.0
    for o, e in zip(counts, exp):
        ao += o
        ae += e
        if ae >= 10:
            obs_m.append(ao)
            exp_m.append(ae)
            ao = ae = 0.0
    if ae > 0:
        obs_m[-1] += ao
        exp_m[-1] += ae
    obs_m, exp_m = np.array(obs_m), np.array(exp_m)
    chi2 = np.sum((obs_m - exp_m) ** 2 / exp_m)
    return stats.chi2.sf(chi2, len(obs_m) - 1), abs(full.sum() - 1.0)


@pytest.mark.parametrize("T", [10.0, 1.0e4])
@pytest.mark.parametrize("x", [0.0, 0.6, 1.0, 1.4, 2.0, 3.0, 4.5, 6.5, 8.8, -2.0])
def test_upar_matches_exact_pdf(O, T, x):
    a = O.damping_a(T)
    u, ntr = O.sample_upar(x, a, 120000, seed=100 + int(T), pid0=10 ** 6)
    assert np.all(ntr >= 1)
    p, norm_err = _chi2_upar(x, a, u)
    assert norm_err < 1e-6          # the binning covers the whole pdf
    assert p > 1e-3


@pytest.mark.parametrize("T", [10.0, 1.0e4])
def test_upar_far_wing_gaussian_is_close(O, T):
    # x >= 9: a Gaussian of mean 1/x, variance 1/2 stands in for Eq. uparf
    a = O.damping_a(T)
    x = 10.0
    u, _ = O.sample_upar(x, a, 120000, seed=5)
    assert np.mean(u) == pytest.approx(1.0 / x, abs=0.01)
    grid = np.linspace(-5, 5, 4001)
    pdf = np.exp(-grid ** 2) / (a * a + (x - grid) ** 2)
    cdf = np.concatenate([[0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    ks = stats.kstest(u, lambda v: np.interp(v, grid, cdf)).statistic
    assert ks < 0.012


@pytest.mark.parametrize("RQ", [0.0, 3.0 / 7.0, 1.0])
def test_phase_inversion_and_moments(O, RQ):
    u = (np.arange(200000) + 0.5) / 200000
    mu = O.sample_mu(RQ, u)
    assert np.all(np.abs(mu) <= 1.0)
    # F(mu) = int_{-1}^{mu} (1 + RQ m^2) dm / int_{-1}^{1} (...): quadrature of Eq. phaseW
    norm = integrate.quad(lambda m: 1 + RQ * m * m, -1, 1)[0]
    for i in range(0, 200000, 9973):
        F = integrate.quad(lambda m: 1 + RQ * m * m, -1, mu[i])[0] / norm
        assert F == pytest.approx(u[i], abs=1e-10)
    m2 = integrate.quad(lambda m: m * m * (1 + RQ * m * m), -1, 1)[0] / norm
    assert np.mean(mu) == pytest.approx(0.0, abs=1e-6)
    assert np.mean(mu * mu) == pytest.approx(m2, abs=1e-5)


def test_phase_moment_values(O):
    # <mu^2> = (1/3 + R/5)/(1 + R/3): 0.4 (wing), 0.3667 (R/Q = 3/7), 0.3556 core mixture
    u = (np.arange(400000) + 0.5) / 400000
    m_w = np.mean(O.sample_mu(1.0, u) ** 2)
    m_c = np.mean(O.sample_mu(3.0 / 7.0, u) ** 2)
    m_i = np.mean(O.sample_mu(0.0, u) ** 2)
    assert m_w == pytest.approx(0.4, abs=1e-5)
    assert m_c == pytest.approx(0.36667, abs=1e-4)
    assert (m_i + 2 * m_c) / 3 == pytest.approx(0.35556, abs=1e-4)


def _scatter_batch(O, n, x, T, atau0, phase=0, g=0.0, seed=3, event=1, rng_dirs=11):
    rng = np.random.default_rng(rng_dirs)
    k = rng.normal(size=(n, 3))
    k /= np.linalg.norm(k, axis=1)[:, None]
    inp = dict(x=np.full(n, x), k=k, a=np.full(n, O.damping_a(T)), g=np.full(n, g),
               atau0=np.full(n, atau0), phase=np.full(n, phase, np.int32),
               pid=np.arange(n, dtype=np.uint64), event=np.full(n, event, np.uint32))
    return inp, O.scatter(inp, seed)


def test_scatter_geometry(O):
    inp, out = _scatter_batch(O, 20000, 1.5, 1e4, -1.0)
    k, kf, ua = inp["k"], out["k_f"], out["u_atom"]
    assert np.allclose(np.linalg.norm(kf, axis=1), 1.0, atol=1e-12)
    assert np.allclose(np.sum(k * kf, axis=1), out["mu"], atol=1e-12)
    assert np.allclose(np.sum(k * ua, axis=1), out["u_par"], atol=1e-12)


@pytest.mark.parametrize("xcrit_target", [0.0, 2.0, 4.0])
def test_core_skip_truncated_gaussian(O, xcrit_target):
    # Sec. 3.2.4: |u_perp| with x_crit has P(|u_perp| > r) = exp(x_crit^2 - r^2), r >= x_crit
    atau0 = (5.0 * xcrit_target) ** 3 if xcrit_target > 0 else -1.0
    inp, out = _scatter_batch(O, 60000, 0.0, 1e4, atau0)
    assert np.allclose(out["x_crit"], xcrit_target, rtol=1e-12)
    uperp = out["u_atom"] - out["u_par"][:, None] * inp["k"]
    r = np.linalg.norm(uperp, axis=1)
    assert np.all(r >= xcrit_target * (1 - 1e-12))
    ks = stats.kstest(r, lambda v: 1.0 - np.exp(np.minimum(xcrit_target ** 2 - v ** 2, 0.0)))
    assert ks.pvalue > 1e-3


def test_core_skip_not_applied_in_wing(O):
    # |x| >= x_crit: no cutoff (Sec. 3.2.4, last sentence before Eq. atau0min)
    inp, out = _scatter_batch(O, 1000, 3.0, 1e4, 1000.0)   # x_crit(1000) = 2 < 3
    assert np.all(out["x_crit"] == 0.0)


def test_phase_choice_frequencies(O):
    T = 1e4
    xcw = O.x_cw_fit(O.damping_a(T))
    _, core = _scatter_batch(O, 60000, 0.5 * xcw, T, -1.0)
    frac0 = np.mean(core["RQ"] == 0.0)
    assert frac0 == pytest.approx(1.0 / 3.0, abs=0.01)
    assert set(np.unique(core["RQ"])) == {0.0, 3.0 / 7.0}
    _, wing = _scatter_batch(O, 1000, 1.2 * xcw, T, -1.0)
    assert np.all(wing["RQ"] == 1.0)
    _, iso = _scatter_batch(O, 1000, 1.2 * xcw, T, -1.0, phase=1)
    assert np.all(iso["RQ"] == 0.0)


def test_recoil_shift(O):
    # Eq. x_f: E[x_f - x + u_par] = E[k_f.u_atom] + g E[mu - 1] = -g for isotropic phase
    g = 0.05
    inp, out = _scatter_batch(O, 200000, 0.3, 1e4, -1.0, phase=1, g=g)
    d = out["x_f"] - inp["x"] + out["u_par"]
    se = np.std(d) / np.sqrt(len(d))
    assert abs(np.mean(d) + g) < 4 * se
    _, out0 = _scatter_batch(O, 200000, 0.3, 1e4, -1.0, phase=1, g=0.0)
    assert np.mean(out["x_f"] - out0["x_f"]) == pytest.approx(-g, rel=0.02)
