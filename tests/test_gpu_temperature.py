"""Temperature suites of uniform slabs (App. "Thermal effects on Ly-alpha
spectra") on the GPU.

Two suites of periodic slabs |z| < H: a fixed line-centre optical depth
tau_0 = 1e7, and a fixed column N_H = 1.7e20 cm^-2, i.e. tau_0 = 1e7 T4^-1/2
(the figure caption's reading: tau_0 = 1e7 at 1e4 K).  Checks:
  * without recoil each spectrum is the Neufeld slab solution (Eq. neufeld) of
    its own a tau_0 wherever a tau_0 >= 1e3 (peaks at 1.066 (a tau_0)^1/3,
    L1 distance < 0.12, as the oracle's analytic test), so the Doppler peak
    moves as T^1/3 (fixed tau_0) and T^1/6 (fixed N_H);
  * with recoil the red peak dominates more and more as T falls (the runaway
    reddening of cold, thick gas the appendix describes), and the GPU spectra
    agree with the oracle's (two-sample chi-square on independent seeds)."""
import numpy as np
import pytest
from scipy import optimize, stats

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu

TS = [10.0, 100.0, 1e3, 1e4]


def _tau0(suite, T):
    return 1e7 if suite == "tau0" else 1e7 * (T / 1e4) ** -0.5


@pytest.fixture(scope="module")
def ctx(colt):
    c = colt.colt_init(0)
    yield c
    colt.colt_finalize(c)


def _gpu(colt, ctx, g, spec):
    h = colt.colt_create_grid(ctx, g)
    try:
        return colt.colt_run(ctx, h, spec)
    finally:
        colt.colt_destroy_grid(ctx, h)


def _peak_coefficient():
    y = optimize.brentq(lambda v: v * np.tanh(v) - 2.0 / 3.0, 1e-6, 10)
    return (y / np.sqrt(np.pi ** 3 / 54.0)) ** (1.0 / 3.0)


@pytest.mark.parametrize("suite", ["tau0", "column"])
def test_recoil_free_suites_follow_neufeld(O, colt, ctx, suite):
    temps = TS + ([1e5] if suite == "tau0" else [])
    for T in temps:
        tau0 = _tau0(suite, T)
        at = O.damping_a(T) * tau0
        assert at >= 1e3
        b = np.sqrt(np.pi ** 3 / 54.0) / at
        J = lambda x: 1.0 / (4 * np.sqrt(6 * np.pi)) * x * x / at / np.cosh(b * x ** 3)
        xp = _peak_coefficient() * at ** (1 / 3)
        L = 3.0 * xp
        spec = S.RunSpec(n_packets=8000, seed=int(120 + T % 97), recoil=False, T_ref=T, spec_units=0,
                         spec_lo=-L, spec_hi=L, spec_nbins=30)
        r = _gpu(colt, ctx, S.slab(16, T, tau0, nxy=2), spec)
        edges = np.linspace(-L, L, 31)
        fine = np.linspace(-L, L, 30001)
        cdf = np.concatenate([[0], np.cumsum(4 * np.pi * J(0.5 * (fine[1:] + fine[:-1])) * np.diff(fine))])
        expected = np.diff(np.interp(edges, fine, cdf))
        got = r["spec"] / r["n_escaped"]
        centres = 0.5 * (edges[1:] + edges[:-1])
        xr = abs(centres[15 + np.argmax(got[15:])])
        xb = abs(centres[np.argmax(got[:15])])
        l1 = 0.5 * np.sum(np.abs(got - expected))
        print(f"{suite} T={T:g} a tau0={at:.3g}: L1 {l1:.3f}, peaks {xr / xp:.2f} {xb / xp:.2f}")
        assert xr == pytest.approx(xp, rel=0.12) and xb == pytest.approx(xp, rel=0.12)
        assert l1 < 0.12


def _asym(spec):
    s = spec.astype(float)
    h = len(s) // 2
    return (s[h:].sum() - s[:h].sum()) / s.sum()


@pytest.mark.parametrize("suite", ["tau0", "column"])
def test_recoil_reddening_grows_as_temperature_falls(O, colt, ctx, suite):
    asym = []
    for T in TS:
        tau0 = _tau0(suite, T)
        g = S.slab(16, T, tau0, nxy=2)
        spec = S.RunSpec(n_packets=8000, seed=140, T_ref=T, spec_units=1, spec_lo=-300.0, spec_hi=300.0,
                         spec_nbins=60)
        rg = _gpu(colt, ctx, g, spec)
        spec.n_packets, spec.seed = 1500, 141
        ro = O.run(g, spec)
        # red = Delta v > 0 (the upper half of the bins)
        asym.append(_asym(rg["spec"]))
        a, b = rg["spec"].astype(float), ro["spec"].astype(float)
        m = (a + b) > 0
        # two-sample chi-square for unequal sample sizes
        k1, k2 = np.sqrt(b.sum() / a.sum()), np.sqrt(a.sum() / b.sum())
        chi2 = np.sum((k1 * a[m] - k2 * b[m]) ** 2 / (a[m] + b[m]))
        p = stats.chi2.sf(chi2, np.count_nonzero(m) - 1)
        print(f"{suite} T={T:g}: red-blue asymmetry GPU {asym[-1]:.3f} oracle {_asym(ro['spec']):.3f}, chi2 p {p:.3g}")
        assert p > 1e-3
        assert rg["n_escaped"] == 8000
    # 10 K > 100 K > 1e3 K (differences of 0.1-0.7 against a noise of 0.011),
    # strongly red at 10 K, nearly symmetric at 1e4 K
    assert asym[0] > asym[1] > asym[2]
    assert asym[0] > (0.3 if suite == "tau0" else 0.6)
    assert abs(asym[3]) < 0.08
