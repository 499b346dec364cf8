"""Pins of the oracle's line constants, Voigt function and crossover frequency
against what the paper and the mathematics fix (no GPU).

Independent references: scipy's Faddeeva function (H = Re w(x + i a)),
erfcx (H(a,0) = e^{a^2} erfc(a)), Dawson's integral (first order in a,
Sec. 3.2.1) and scipy's Lambert W (Sec. 3.2.2)."""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import dawsn, erfcx, lambertw, wofz

PC = 3.0856775814913673e18
TS = [1.0, 10.0, 100.0, 1.0e3, 1.0e4, 1.0e5]


def test_line_constants_match_printed_coefficients(O, paper):
    c = paper["line_constants"]
    assert O.vth_kms(1e4) == pytest.approx(c["vth_kms_T4_1"], rel=1e-12)
    assert O.damping_a(1e4) == pytest.approx(c["a_T4_1"], rel=1e-12)
    assert O.sigma0(1e4) == pytest.approx(c["sigma0_T4_1_cm2"], rel=1e-12)
    assert O.recoil_g(1e4) == pytest.approx(c["recoil_g_T4_1"], rel=1e-12)
    # T scalings: v_th ~ T^1/2, a, sigma_0, g ~ T^-1/2
    assert O.vth_kms(100.0) == pytest.approx(12.85 / 10.0, rel=1e-12)
    assert O.damping_a(100.0) == pytest.approx(4.702e-4 * 10.0, rel=1e-12)
    # Eq. tauH: n sigma_0 (1 pc) = 1.820e5 at T4 = 1
    assert O.sigma0(1e4) * PC == pytest.approx(c["tauH_coefficient_per_cm3_pc"], rel=2e-3)
    # Eq. atau0min: a sigma_0 (1 pc) = 85.56 at T4 = 1
    assert O.damping_a(1e4) * O.sigma0(1e4) * PC == pytest.approx(paper["atau0_local_coefficient"]["value"], rel=2e-3)
    # Eq. recoil: g ~ 0.54 a
    assert O.recoil_g(1e4) / O.damping_a(1e4) == pytest.approx(c["recoil_g_over_a"], abs=0.005)
    # Eq. atau0J: with the Jeans length 0.75 kpc T4^1/2 n^-1/2 and a sigma_0 from Sec. 2
    aj = paper["atau0_jeans"]
    atau_j = O.damping_a(1e4) * O.sigma0(1e4) * 1.0 * 750.0 * PC
    assert atau_j == pytest.approx(aj["coefficient"], rel=2e-3)
    assert O.x_crit(atau_j) == pytest.approx(aj["x_crit_T1e4_n1"], abs=0.05)


@pytest.mark.parametrize("T", TS)
def test_H_exact_equals_faddeeva(O, T):
    a = O.damping_a(T)
    x = np.concatenate([np.linspace(0.0, 12.0, 481), np.geomspace(12.0, 3.0e3, 60)])
    he = O.H_exact(a, x)
    hw = wofz(x + 1j * a).real
    assert np.max(np.abs(he / hw - 1.0)) < 1e-9


@pytest.mark.parametrize("a", [1e-4, 1e-2, 0.3])
def test_H_exact_closed_form_at_line_centre(O, a):
    assert O.H_exact(a, 0.0) == pytest.approx(erfcx(a), rel=1e-11)


@pytest.mark.parametrize("a", [4.702e-4, 0.0149])
def test_H_exact_normalisation(O, a):
    # int H dx = sqrt(pi): quadrature out to X plus the a/(sqrt(pi) x^2) tail
    X = 2000.0
    f = lambda x: float(O.H_exact(a, x))
    pts = [0.5, 1, 2, 3, 4, 6, 10, 30, 100, 300]
    core, _ = integrate.quad(f, 0.0, X, points=pts, limit=400, epsabs=0, epsrel=1e-11)
    tail = a / (np.sqrt(np.pi) * X) * (1 + 0.5 / X ** 2)
    assert 2.0 * (core + tail) == pytest.approx(np.sqrt(np.pi), rel=1e-8)


@pytest.mark.parametrize("T", [1.0, 10.0, 100.0, 1.0e3, 1.0e4])
def test_H_approx_within_one_per_cent(O, paper, T):
    a = O.damping_a(T)
    x = np.linspace(0.0, 60.0, 6001)
    err = np.abs(O.H_approx(a, x) / wofz(x + 1j * a).real - 1.0)
    assert np.max(err) < paper["H_approx"]["max_rel_error"]


def test_H_approx_improves_with_temperature(O):
    x = np.linspace(0.0, 60.0, 6001)
    errs = []
    for T in [1.0, 10.0, 100.0, 1.0e4]:
        a = O.damping_a(T)
        errs.append(np.max(np.abs(O.H_approx(a, x) / wofz(x + 1j * a).real - 1.0)))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[-1] < 2e-5


def test_H_approx_first_order_term_is_dawson(O):
    # Sec. 3.2.1: H = e^{-x^2} + (2a/sqrt(pi)) (2 x F(x) - 1) + O(a^2); the
    # approximation keeps first order, so its a-coefficient must match this
    # (tiny a isolates it).  A wrong Table AB coefficient breaks this.
    a = 1e-7
    regions = [(np.linspace(0.0, np.sqrt(3.0), 300), 2e-3),
               (np.linspace(np.sqrt(3.0) * (1 + 1e-9), 5.0 * (1 - 1e-9), 300), 2e-4)]
    for x, tol in regions:
        coef = (O.H_approx(a, x) - np.exp(-x * x)) / a
        exact = (2.0 / np.sqrt(np.pi)) * (2.0 * x * dawsn(x) - 1.0)
        assert np.max(np.abs(coef / exact - 1.0)) < tol
    # wing (z >= 25): the approximation drops exp(-z) < 1.4e-11, so compare the
    # whole first-order H at an a where that term is negligible
    a = 1e-4
    x = np.geomspace(5.0, 300.0, 300)
    exact = np.exp(-x * x) + a * (2.0 / np.sqrt(np.pi)) * (2.0 * x * dawsn(x) - 1.0)
    assert np.max(np.abs(O.H_approx(a, x) / exact - 1.0)) < 1e-3


def test_H_approx_continuity_at_region_edges(O):
    for T in [10.0, 1.0e4]:
        a = O.damping_a(T)
        for z in (3.0, 25.0):
            x = np.sqrt(z)
            lo = O.H_approx(a, x * (1 - 1e-12))
            hi = O.H_approx(a, x * (1 + 1e-12))
            assert abs(hi / lo - 1.0) < 2e-4


def test_H_approx_wing_asymptote(O):
    a = 4.702e-4
    x = np.geomspace(10.0, 1e4, 50)
    asym = a / (np.sqrt(np.pi) * x * x) * (1 + 1.5 / x ** 2 + 15.0 / (4 * x ** 4))
    assert np.max(np.abs(O.H_approx(a, x) / asym - 1.0)) < 1e-3


def test_x_cw_lambert_matches_library(O):
    for T in TS:
        a = O.damping_a(T)
        w = lambertw(-a / np.sqrt(np.pi), -1).real
        assert O.x_cw_lambert(a) == pytest.approx(np.sqrt(-w), rel=1e-12)
        # the crossover solves exp(-x^2) = a / (sqrt(pi) x^2)
        xc = O.x_cw_lambert(a)
        assert np.exp(-xc * xc) == pytest.approx(a / (np.sqrt(np.pi) * xc * xc), rel=1e-10)


def test_x_cw_fit_accuracy(O, paper):
    Ts = np.geomspace(*paper["x_cw_fit"]["T_range_K"], 60)
    errs = [abs(O.x_cw_fit(O.damping_a(T)) / O.x_cw_lambert(O.damping_a(T)) - 1.0) for T in Ts]
    assert max(errs) < paper["x_cw_fit"]["max_rel_error"]
    # natural log in the fit: the value at T = 1e4 K is ~3.25
    assert O.x_cw_fit(4.702e-4) == pytest.approx(3.254, abs=2e-3)


def test_x_crit_values(O, paper):
    xc = paper["x_crit"]
    assert O.x_crit(xc["atau0"][0]) == pytest.approx(xc["x_crit"][0], rel=1e-12)
    assert O.x_crit(xc["atau0"][1]) == pytest.approx(xc["x_crit"][1], abs=0.05)
    assert O.x_crit(0.999) == 0.0
    assert O.x_crit(8.0e3) == pytest.approx(4.0, rel=1e-12)
