"""The oracle's exact-physics mode (no GPU): H(a,x) by quadrature instead of
H_approx and the far-wing u_par by numeric inversion of Eq. uparf instead of
the Gaussian, used to measure the bias of the approximations.

  * the exact far-wing sampler follows Eq. uparf (histogram against the
    distribution integrated by adaptive quadrature, chi-square), where the
    Gaussian of mean 1/|x| is only close;
  * a static sphere solved exactly (no core-skipping, exact H and wing) and
    with the approximations (core-skipping on) emits the same spectrum
    (two-sample chi-square on independent seeds)."""
import numpy as np
import pytest
from scipy import integrate, stats
from scipy.special import wofz

from paper_1409_4480_gb300 import synth as S


def _bin_probs(x, a, edges):
    f = lambda u: np.exp(-u * u) / ((x - u) ** 2 + a * a)
    tot = integrate.quad(f, -10, 10, epsabs=0, epsrel=1e-12, limit=200)[0]
    return np.array([integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-12)[0]
                     for lo, hi in zip(edges[:-1], edges[1:])]) / tot


@pytest.mark.parametrize("x,a", [(9.5, 0.0149), (20.0, 4.702e-4), (-12.0, 0.0149)])
def test_exact_far_wing_sampler_follows_eq_uparf(O, x, a):
    n = 20000
    u, ntr = O.sample_upar(x, a, n, seed=91, exact=True)
    assert np.all(ntr == 1)
    edges = np.linspace(-3.0, 3.0, 31)
    p = _bin_probs(x, a, edges)
    counts = np.histogram(u, bins=edges)[0].astype(float)
    m = n * p > 5
    chi2 = np.sum((counts[m] - n * p[m]) ** 2 / (n * p[m]))
    assert stats.chi2.sf(chi2, np.count_nonzero(m) - 1) > 1e-3
    # the exact mean against the one from quadrature
    mean = integrate.quad(lambda v: v * np.exp(-v * v) / ((x - v) ** 2 + a * a), -10, 10, epsrel=1e-12)[0] / \
        integrate.quad(lambda v: np.exp(-v * v) / ((x - v) ** 2 + a * a), -10, 10, epsrel=1e-12)[0]
    assert abs(u.mean() - mean) < 4 * u.std() / np.sqrt(n)
    # the default mode's Gaussian is centred on 1/x, not on the exact mean
    ug, _ = O.sample_upar(x, a, n, seed=91)
    print(f"x={x}: exact mean {mean:.5f}, 1/x = {1 / x:.5f}, sampled exact {u.mean():.5f}, Gaussian {ug.mean():.5f}")


def test_exact_and_approximate_spectra_agree(O):
    # static dust-free sphere, T = 10 K, tau0 = 1e3 (a tau0 = 15), recoil off
    g = S.sphere(8, 10.0, 1e3)
    spec = S.RunSpec(n_packets=1000, seed=93, recoil=False, core_skip=0, albedo=0.0, T_ref=10.0, spec_units=0,
                     spec_lo=-12.0, spec_hi=12.0, spec_nbins=24)
    ex = O.run(g, spec, exact=True)
    spec.core_skip, spec.seed = 1, 94
    ap = O.run(g, spec)
    assert ex["n_escaped"] == 1000 and ap["n_escaped"] == 1000
    a, b = ex["spec"].astype(float), ap["spec"].astype(float)
    m = (a + b) > 0
    chi2 = np.sum((a[m] - b[m]) ** 2 / (a[m] + b[m]))
    assert stats.chi2.sf(chi2, np.count_nonzero(m) - 1) > 1e-3
    # the quadrature H the exact mode evaluates is the Faddeeva value (here at line centre)
    assert np.real(wofz(1j * 0.0149)) == pytest.approx(O.H_exact(0.0149, 0.0), rel=1e-10)


@pytest.mark.parametrize("x,a", [(9.0, 0.0149), (12.0, 4.702e-4), (30.0, 0.0149)])
def test_far_wing_gaussian_ks_distance(O, x, a):
    # Sec. 3.2.3 replaces Eq. uparf beyond |x| = 9 by a Gaussian of mean 1/|x|;
    # its Kolmogorov-Smirnov distance to the exact distribution (reported) is
    # within the sampling noise of 4e4 draws, ~0.005-0.01, from |x| = 9 on
    grid = np.linspace(-6.0, 6.0, 24001)
    f = np.exp(-grid ** 2) / ((x - grid) ** 2 + a * a)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    exact_cdf = lambda u: np.interp(u, grid, cdf)
    n = 40000
    ug, _ = O.sample_upar(x, a, n, seed=95)
    d_gauss = stats.kstest(ug, exact_cdf).statistic
    ue, _ = O.sample_upar(x, a, n, seed=96, exact=True)
    d_exact = stats.kstest(ue, exact_cdf).statistic
    print(f"x={x}: KS distance, Gaussian {d_gauss:.4f}, exact sampler {d_exact:.4f}")
    assert d_gauss < 0.02
    assert stats.kstest(ue, exact_cdf).pvalue > 1e-3
