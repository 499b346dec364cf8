"""Pins of the oracle's diffuse emission and Jeans core-skipping (no GPU).

Diffuse emission (Sec. 3.1.1: recombination and collisional excitation emit
from the gas itself): a packet starts in cell c with probability proportional
to its luminosity, at a uniform position in the cell, with an isotropic
direction.  In an empty box every packet escapes unscattered with weight 1,
so a camera image counts where packets were born: its pixel sums must follow
the multinomial law of the column luminosities, exactly zero where no cell
emits.  The Jeans estimate (Eq. atau0J) is pinned to the Jeans length computed
from physical constants and to the paper's x_crit,J ~ 8 (T = 1e4 K, n = 1)."""
import numpy as np
import pytest
from scipy import stats

from paper_1409_4480_gb300 import synth as S

K_B = 1.380649e-16       # erg / K
G_N = 6.67430e-8         # cm^3 g^-1 s^-2
M_H = 1.6735575e-24      # g (hydrogen atom)
KPC = 3.0856775814913673e21


def _jeans_length(T, n):
    # lambda_J = sqrt(15 k T / (4 pi G mu rho)), mu = 1.23 m_H, rho = m_H n / X, X = 0.75 (Sec. 3.2.4)
    mu, rho = 1.23 * M_H, M_H * n / 0.75
    return np.sqrt(15.0 * K_B * T / (4.0 * np.pi * G_N * mu * rho))


def test_jeans_length_printed_value(paper):
    # the paper's 0.75 kpc T4^1/2 n^-1/2 from the definition
    assert _jeans_length(1e4, 1.0) / KPC == pytest.approx(0.75, rel=5e-3)


@pytest.mark.parametrize("T,n", [(1e4, 1.0), (100.0, 1.0), (1e4, 1e-3), (3e3, 50.0), (1e5, 0.2)])
def test_atau_jeans_from_the_jeans_length(O, T, n):
    # a tau_J = a sigma_0 n lambda_J over a uniform region one Jeans length across
    expect = O.damping_a(T) * O.sigma0(T) * n * _jeans_length(T, n)
    assert O.atau_jeans(T, n) == pytest.approx(expect, rel=4e-3)


def test_x_crit_jeans_printed(O, paper):
    aj = paper["atau0_jeans"]
    assert O.x_crit(O.atau_jeans(1e4, 1.0)) == pytest.approx(aj["x_crit_T1e4_n1"], abs=0.05)
    assert O.atau_jeans(0.0 + 1e4, 0.0) == 0.0


def _thin_box(shape, lum, npix_cam=None):
    lo, hi = (-1e18,) * 3, (1e18,) * 3
    g = S.uniform_box(shape, lo, hi, 0.0, 1e4)
    g.lum = np.asarray(lum, np.float64)
    return g


def _image_counts(r, spec, shape):
    # the image of one camera, summed over frequency: [v][u]
    npix = spec.cameras[0].npix
    img = r["cam_image"].reshape(npix, npix, spec.cam_nbins).sum(axis=2)
    return img


def test_diffuse_thin_box_follows_the_luminosity(O):
    rng = np.random.default_rng(7)
    shape = (6, 6, 6)
    lum = rng.lognormal(0.0, 1.0, size=216)
    lum[rng.random(216) < 0.2] = 0.0                   # dark cells never emit
    g = _thin_box(shape, lum)
    N = 60000
    spec = S.RunSpec(n_packets=N, seed=71, source=1, spec_units=0, spec_lo=-1, spec_hi=1, spec_nbins=2,
                     cameras=S.axis_cameras(6, ("+z",)), cam_units=0, cam_lo=-1, cam_hi=1, cam_nbins=2)
    r = O.run(g, spec, images=True)
    assert r["n_escaped"] == N and r["n_scat"] == 0
    # camera +z: image axes (e_x, e_y), image[v][u]; pixel (u, v) = (i, j) sees the column of cells (i, j)
    img = _image_counts(r, spec, shape)
    col = lum.reshape(6, 6, 6).sum(axis=0)            # [j, i] summed over k
    expect = N * col / col.sum()
    dark = expect == 0
    assert np.all(img[dark] == 0)
    chi2 = np.sum((img[~dark] - expect[~dark]) ** 2 / expect[~dark])
    assert stats.chi2.sf(chi2, np.count_nonzero(~dark) - 1) > 1e-3
    # every packet leaves at x = 0 with weight exp(-0) = 1
    assert r["cam_total"][0] == pytest.approx(N, rel=1e-12)


def test_diffuse_single_bright_cell_and_uniform_position(O):
    # one emitting cell: all packets start there; inside it the position is
    # uniform, so a camera with 8x8 pixels over that cell sees a flat image
    shape = (3, 3, 3)
    lum = np.zeros(27)
    lum[13] = 2.5                                      # the centre cell (1, 1, 1)
    g = _thin_box(shape, lum)
    h = (2e18) / 3.0
    N = 32000
    spec = S.RunSpec(n_packets=N, seed=72, source=1, spec_units=0, spec_lo=-1, spec_hi=1, spec_nbins=1,
                     cameras=S.axis_cameras(8, ("+x",)), cam_units=0, cam_lo=-1, cam_hi=1, cam_nbins=1,
                     fov_half=0.5 * h)
    r = O.run(g, spec, images=True)
    img = r["cam_image"].reshape(8, 8)
    assert img.sum() == N
    chi2 = np.sum((img - N / 64.0) ** 2 / (N / 64.0))
    assert stats.chi2.sf(chi2, 63) > 1e-3


def test_diffuse_two_cell_probabilities(O):
    # luminosities 1 : 3 -> starting-cell probabilities 1/4 : 3/4 (binomial)
    g = S.uniform_box((2, 1, 1), (-1e18,) * 3, (1e18,) * 3, 0.0, 1e4)
    g.lum = np.array([1.0, 3.0])
    N = 40000
    spec = S.RunSpec(n_packets=N, seed=73, source=1, spec_units=0, spec_lo=-1, spec_hi=1, spec_nbins=1,
                     cameras=S.axis_cameras(2, ("+z",)), cam_units=0, cam_lo=-1, cam_hi=1, cam_nbins=1)
    r = O.run(g, spec, images=True)
    img = r["cam_image"].reshape(2, 2)                 # [v = y][u = x]
    assert img.sum() == N
    assert abs(img[:, 0].sum() - N / 4) <= 4 * np.sqrt(N * 0.25 * 0.75)


def test_diffuse_octree_follows_the_luminosity(O):
    # octree leaves of mixed size: pixel counts follow the projected luminosity
    base = S.uniform_box((8, 8, 8), (-1e18,) * 3, (1e18,) * 3, 0.0, 1e4)
    g = S.octree_from_cartesian(base, seed=5)
    rng = np.random.default_rng(9)
    lum = rng.random(g.n_cells) * (rng.random(g.n_cells) < 0.7)
    g.lum = lum
    N = 50000
    spec = S.RunSpec(n_packets=N, seed=74, source=1, spec_units=0, spec_lo=-1, spec_hi=1, spec_nbins=1,
                     cameras=S.axis_cameras(8, ("+z",)), cam_units=0, cam_lo=-1, cam_hi=1, cam_nbins=1)
    r = O.run(g, spec, images=True)
    assert r["n_escaped"] == N
    img = r["cam_image"].reshape(8, 8)
    # expected: each leaf spreads its luminosity evenly over the pixels it covers
    lv = g.leaf_level.astype(int)
    ijk = g.leaf_ijk.reshape(-1, 3).astype(np.int64)
    expect = np.zeros((8, 8))
    for c in range(g.n_cells):
        s = 8 >> lv[c]                                  # pixels per leaf side (finest level 3)
        i0, j0 = ijk[c, 0] * s, ijk[c, 1] * s
        expect[j0:j0 + s, i0:i0 + s] += lum[c] / (s * s)
    expect *= N / lum.sum()
    m = expect > 0
    assert np.all(img[~m] == 0)
    chi2 = np.sum((img[m] - expect[m]) ** 2 / expect[m])
    assert stats.chi2.sf(chi2, np.count_nonzero(m) - 1) > 1e-3


def test_diffuse_rejects_bad_luminosities(O):
    g = S.uniform_box((2, 2, 2), (-1.0,) * 3, (1.0,) * 3, 0.0, 1e4)
    spec = S.RunSpec(n_packets=10, seed=1, source=1)
    for bad in (np.zeros(8), -np.ones(8), np.full(8, np.nan)):
        g.lum = bad
        with pytest.raises(ValueError):
            O.run(g, spec)
    g.lum = None
    with pytest.raises(ValueError):
        O.run(g, spec)


def test_jeans_core_skip_keeps_the_spectrum(O):
    # a static uniform sphere several Jeans lengths across (a tau_0 = 2 a tau_J):
    # core-skipping with the Jeans estimate (x_crit,J = 1.7) and with the cell +
    # non-local estimate give the same emergent spectrum (two-sample chi-square),
    # and the Jeans estimate skips more scatterings
    T, n = 1e4, 1e-4
    lam = _jeans_length(T, n)
    R = 2.0 * lam
    tau0 = n * O.sigma0(T) * R
    g = S.sphere(12, T, tau0, R=R)
    xp = 0.931 * (O.damping_a(T) * tau0) ** (1 / 3)
    L = 3.0 * xp
    runs = []
    for mode, seed in ((1, 81), (2, 82)):
        spec = S.RunSpec(n_packets=1500, seed=seed, recoil=False, core_skip=mode, albedo=0.0,
                         spec_lo=-L, spec_hi=L, spec_nbins=20)
        runs.append(O.run(g, spec))
    a, b = (r["spec"].astype(float) for r in runs)
    assert runs[0]["n_escaped"] == 1500 and runs[1]["n_escaped"] == 1500
    m = (a + b) > 0
    chi2 = np.sum((a[m] - b[m]) ** 2 / (a[m] + b[m]))
    assert stats.chi2.sf(chi2, np.count_nonzero(m) - 1) > 1e-3
    assert runs[1]["n_scat"] < runs[0]["n_scat"]


def test_diffuse_natural_emission_mixes_the_cells_voigt_profiles(O):
    # diffuse natural + thermal emission from an empty box of two cells at
    # 100 K and 1e4 K with luminosities 1 : 3: every packet leaves unscattered
    # with the frequency it was born with, so the escape spectrum in Delta v is
    # the luminosity-weighted mix of the two cells' Voigt profiles, each
    # H(a,x)/sqrt(pi) in x = -Delta v / v_th (exact H from the Faddeeva function)
    from scipy.special import wofz
    g = S.uniform_box((2, 1, 1), (-1e18,) * 3, (1e18,) * 3, 1e-30, 1e4)
    g.T = np.array([100.0, 1e4], np.float32)
    g.lum = np.array([1.0, 3.0])
    N = 80000
    edges = np.linspace(-60.0, 60.0, 61)
    spec = S.RunSpec(n_packets=N, seed=75, source=1, emission=1, spec_units=1, spec_lo=-60.0, spec_hi=60.0,
                     spec_nbins=60)
    r = O.run(g, spec)
    assert r["n_escaped"] == N and r["n_scat"] == 0
    v = np.linspace(-60.0, 60.0, 60 * 200 + 1)
    p = np.zeros_like(v)
    for T, w in ((100.0, 0.25), (1e4, 0.75)):
        vth, a = O.vth_kms(T), O.damping_a(T)
        p += w * np.real(wofz(-v / vth + 1j * a)) / np.sqrt(np.pi) / vth
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (p[1:] + p[:-1]) * np.diff(v))])
    p_bins = np.diff(np.interp(edges, v, cdf))
    counts = r["spec"].astype(float)
    m = p_bins * N > 5
    chi2 = np.sum((counts[m] - N * p_bins[m]) ** 2 / (N * p_bins[m]))
    assert stats.chi2.sf(chi2, np.count_nonzero(m) - 1) > 1e-3


def test_several_point_sources_in_proportion_to_their_weights(O):
    # an empty box: every packet leaves unscattered, and its emission peel-off
    # (weight 1, no attenuation) lands in the pixel of the source it was born
    # at; the sources' shares of the image follow their weights (binomial),
    # and a source of weight 0 never emits
    g = S.uniform_box((4, 4, 4), (-4e18,) * 3, (4e18,) * 3, 1e-30, 1e4)
    pos = [(-3e18, -3e18, 0.0), (1e18, -3e18, 0.0), (-3e18, 1e18, 0.0), (3e18, 3e18, 0.0)]
    w = [1.0, 2.0, 5.0, 0.0]
    N = 40000
    spec = S.RunSpec(n_packets=N, seed=17, spec_units=1, spec_lo=-50, spec_hi=50, spec_nbins=10,
                     cameras=S.axis_cameras(8, ("+z",)), cam_units=1, cam_lo=-50, cam_hi=50, cam_nbins=1,
                     sources=[(p, 0.0, wi) for p, wi in zip(pos, w)])
    r = O.run(g, spec, images=True)
    img = r["cam_image"].reshape(8, 8)                      # [v][u]; u = +x, v = +y for the +z camera
    pix = lambda p: (int((p[1] + 4e18) / 1e18), int((p[0] + 4e18) / 1e18))
    got = np.array([img[pix(p)] for p in pos])
    assert got.sum() == pytest.approx(N) and got[3] == 0
    for k in range(3):
        f = w[k] / sum(w)
        assert abs(got[k] - N * f) < 4 * np.sqrt(N * f * (1 - f)), (k, got)


def test_one_listed_source_equals_the_single_source(O):
    g = S.sphere(16, 1e4, 1e5, v_max_kms=50.0, tau_dust=0.5)
    base = S.RunSpec(n_packets=600, seed=9, src_pos=(2e17, -1e17, 3e17), src_sigma=1e17, albedo=0.32,
                     spec_units=1, spec_lo=-300, spec_hi=300, spec_nbins=30, max_scatter=50)
    a = O.run(g, base, per_packet=True)
    b = O.run(g, S.RunSpec(**{**base.__dict__, "src_pos": (0.0, 0.0, 0.0), "src_sigma": 0.0,
                              "sources": [((2e17, -1e17, 3e17), 1e17, 3.0)]}), per_packet=True)
    for k in ("pk_status", "pk_nscat", "pk_freq", "spec"):
        assert np.array_equal(a[k], b[k])
