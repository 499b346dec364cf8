"""GPU parity of diffuse emission and Jeans core-skipping against the oracle.

Diffuse emission picks the starting cell with integer arithmetic on both
sides (a 64-bit Philox word times the total weight, then a search of the
prefix sums), so in an empty box, where every packet leaves unscattered with
weight exactly 1 and pixel edges fall on cell faces, the camera images are
compared bit for bit.  With gas, 20-scattering prefixes are compared packet
by packet as for point sources.  The Jeans estimate (Eq. atau0J) changes only
a tau_0 of the scattering, so prefixes are compared packet by packet and full
histories statistically."""
import numpy as np
import pytest
from scipy import stats

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu

PREFIX = 20
FTOL = 1e-3
MIN_SAME = 0.98
MIN_DISCRETE = 0.99


@pytest.fixture(scope="module")
def ctx(colt):
    c = colt.colt_init(0)
    yield c
    colt.colt_finalize(c)


def _run_both(O, colt, ctx, g, spec, precision, per_packet=True, images=False):
    spec.precision = precision
    h = colt.colt_create_grid(ctx, g, f_nl=spec.f_nl)
    try:
        rg = colt.colt_run(ctx, h, spec, per_packet=per_packet, images=images)
    finally:
        colt.colt_destroy_grid(ctx, h)
    ro = O.run(g, spec, per_packet=per_packet, images=images)
    return rg, ro


def _identity(rg, ro):
    same = (rg["pk_status"] == ro["pk_status"]) & (rg["pk_nscat"] == ro["pk_nscat"])
    fclose = np.abs(rg["pk_freq"] - ro["pk_freq"]) <= FTOL * np.maximum(1.0, np.abs(ro["pk_freq"]))
    full, disc = np.mean(same & fclose), np.mean(same)
    assert disc >= MIN_DISCRETE, disc
    return full


def _same_images(rg, ro, precision, N):
    # pixel edges lie on cell faces and a position is at least 2^-24 cell
    # widths from a face, so FP64 pixel arithmetic cannot move a packet: the
    # images agree bit for bit.  FP32 pixel arithmetic (mixed precision) may
    # move a packet within a few FP32 ulps of a face to the next pixel.
    if precision == 0:
        assert np.array_equal(rg["cam_image"], ro["cam_image"])
    else:
        assert rg["cam_image"].sum() == ro["cam_image"].sum()
        assert np.abs(rg["cam_image"] - ro["cam_image"]).sum() <= 2e-4 * N * 6


def _thin(shape, lum):
    g = S.uniform_box(shape, (-1e18,) * 3, (1e18,) * 3, 0.0, 1e4)
    g.lum = np.asarray(lum, np.float64)
    return g


@pytest.mark.parametrize("precision", [0, 1])
def test_diffuse_thin_box_images(O, colt, ctx, precision):
    rng = np.random.default_rng(101)
    shape = (16, 12, 10)                       # ragged
    n = 16 * 12 * 10
    lum = rng.lognormal(0.0, 2.0, n) * (rng.random(n) < 0.8)
    g = _thin(shape, lum)
    N = 200000
    cams = [S.Camera((0.0, 0.0, 1.0), 16), S.Camera((1.0, 0.0, 0.0), 12), S.Camera((0.0, -1.0, 0.0), 16)]
    spec = S.RunSpec(n_packets=N, seed=102, source=1, spec_units=0, spec_lo=-1, spec_hi=1, spec_nbins=2,
                     cameras=cams, cam_units=0, cam_lo=-1, cam_hi=1, cam_nbins=2, fov_half=1e18)
    rg, ro = _run_both(O, colt, ctx, g, spec, precision, per_packet=False, images=True)
    assert rg["n_escaped"] == N and rg["n_scat"] == 0
    assert np.array_equal(rg["cam_spec"], ro["cam_spec"])
    _same_images(rg, ro, precision, N)


def test_diffuse_octree_images(O, colt, ctx):
    base = S.uniform_box((16, 16, 16), (-1e18,) * 3, (1e18,) * 3, 0.0, 1e4)
    g = S.octree_from_cartesian(base, seed=103)
    rng = np.random.default_rng(104)
    g.lum = rng.random(g.n_cells) ** 3 * (rng.random(g.n_cells) < 0.9)
    N = 100000
    spec = S.RunSpec(n_packets=N, seed=105, source=1, spec_units=0, spec_lo=-1, spec_hi=1, spec_nbins=1,
                     cameras=S.axis_cameras(16, ("+z", "-x")), cam_units=0, cam_lo=-1, cam_hi=1, cam_nbins=1)
    for precision in (0, 1):
        rg, ro = _run_both(O, colt, ctx, g, spec, precision, per_packet=False, images=True)
        assert rg["n_escaped"] == N
        _same_images(rg, ro, precision, N)


@pytest.mark.parametrize("precision", [0, 1])
def test_diffuse_dusty_outflow_prefix_identity(O, colt, ctx, precision):
    # a dusty Hubble-flow sphere emitting in proportion to n^2 (recombination-like)
    g = S.sphere(32, 1e4, 1e5, v_max_kms=200.0, tau_dust=1.0)
    g.lum = np.asarray(g.n_HI, np.float64) ** 2
    spec = S.RunSpec(n_packets=3000, seed=106, source=1, albedo=0.32, max_scatter=PREFIX, spec_units=1,
                     spec_lo=-1000, spec_hi=1000, spec_nbins=200, cameras=S.axis_cameras(16), cam_units=1,
                     cam_lo=-1000, cam_hi=1000, cam_nbins=200)
    rg, ro = _run_both(O, colt, ctx, g, spec, precision, images=True)
    assert rg["n_emitted"] == 3000
    assert rg["n_escaped"] + rg["n_absorbed"] + rg["n_capped"] == 3000
    assert _identity(rg, ro) >= MIN_SAME
    tol = 0.002 if precision == 0 else 0.03
    assert np.sum(np.abs(rg["cam_spec"] - ro["cam_spec"])) <= tol * np.sum(ro["cam_spec"])


def test_diffuse_natural_emission_octree_prefix(O, colt, ctx):
    g = S.octree_sphere(1e4, 1e5, v_max_kms=-100.0, tau_dust=0.5)
    g.lum = np.asarray(g.n_HI, np.float64) * (1.0 + np.arange(g.n_cells) % 3)
    spec = S.RunSpec(n_packets=3000, seed=107, source=1, emission=1, max_scatter=PREFIX, spec_units=1,
                     spec_lo=-1000, spec_hi=1000, spec_nbins=100)
    for precision in (0, 1):
        rg, ro = _run_both(O, colt, ctx, g, spec, precision)
        assert _identity(rg, ro) >= MIN_SAME


def test_diffuse_argument_errors(colt, ctx):
    g = S.uniform_box((2, 2, 2), (-1.0,) * 3, (1.0,) * 3, 1.0, 1e4)
    h = colt.colt_create_grid(ctx, g)
    try:
        spec = S.RunSpec(n_packets=10, seed=1, source=1)
        with pytest.raises(colt.ColtError):           # no luminosity set
            colt.colt_run(ctx, h, spec)
        for bad in (np.zeros(8), -np.ones(8), np.full(8, np.inf)):
            with pytest.raises(colt.ColtError):
                colt.colt_set_cell_luminosity(ctx, h, bad)
        colt.colt_set_cell_luminosity(ctx, h, np.ones(8))
        r = colt.colt_run(ctx, h, spec)
        assert r["n_emitted"] == 10
        spec.source = 7
        with pytest.raises(colt.ColtError):
            colt.colt_run(ctx, h, spec)
        spec.source, spec.core_skip = 0, 3
        with pytest.raises(colt.ColtError):
            colt.colt_run(ctx, h, spec)
    finally:
        colt.colt_destroy_grid(ctx, h)


def test_diffuse_luminosity_from_device_memory(colt, ctx):
    torch = pytest.importorskip("torch")
    g = _thin((4, 4, 4), np.ones(64))
    lum = np.random.default_rng(3).random(64)
    spec = S.RunSpec(n_packets=5000, seed=108, source=1, spec_units=0, spec_lo=-1, spec_hi=1, spec_nbins=1,
                     cameras=S.axis_cameras(4, ("+z",)), cam_units=0, cam_lo=-1, cam_hi=1, cam_nbins=1)
    out = []
    for src in ("host", "device"):
        g.lum = None
        h = colt.colt_create_grid(ctx, g)
        try:
            colt.colt_set_cell_luminosity(ctx, h, lum if src == "host" else torch.tensor(lum, device="cuda"))
            out.append(colt.colt_run(ctx, h, spec, images=True)["cam_image"])
        finally:
            colt.colt_destroy_grid(ctx, h)
    assert np.array_equal(out[0], out[1])


def _jeans_sphere():
    T, n = 1e4, 1e-4
    lam = 0.75 * 3.0856775814913673e21 * np.sqrt(T / 1e4) / np.sqrt(n)
    R = 2.0 * lam
    tau0 = n * 5.898e-14 * R
    return S.sphere(24, T, tau0, R=R, tau_dust=0.3)


@pytest.mark.parametrize("precision", [0, 1])
def test_jeans_prefix_identity(O, colt, ctx, precision):
    g = _jeans_sphere()
    spec = S.RunSpec(n_packets=3000, seed=109, core_skip=2, max_scatter=PREFIX, spec_units=1, spec_lo=-300,
                     spec_hi=300, spec_nbins=60)
    rg, ro = _run_both(O, colt, ctx, g, spec, precision)
    assert _identity(rg, ro) >= MIN_SAME


def test_jeans_full_histories_statistics(O, colt, ctx):
    g = _jeans_sphere()
    N = 4000
    spec = S.RunSpec(n_packets=N, seed=110, core_skip=2, albedo=0.32, spec_units=1, spec_lo=-300, spec_hi=300,
                     spec_nbins=30)
    spec.precision = 1
    h = colt.colt_create_grid(ctx, g)
    try:
        rg = colt.colt_run(ctx, h, spec)
    finally:
        colt.colt_destroy_grid(ctx, h)
    spec.seed = 111
    ro = O.run(g, spec)
    f1, f2 = rg["n_escaped"] / N, ro["n_escaped"] / N
    f = 0.5 * (f1 + f2)
    assert abs(f1 - f2) <= 3.5 * np.sqrt(f * (1 - f) * 2.0 / N) + 1e-12
    a, b = rg["spec"].astype(float), ro["spec"].astype(float)
    a, b = a / a.sum() * (a.sum() + b.sum()) / 2, b / b.sum() * (a.sum() + b.sum()) / 2
    m = (a + b) > 0
    chi2 = np.sum((a[m] - b[m]) ** 2 / (a[m] + b[m]))
    assert stats.chi2.sf(chi2, np.count_nonzero(m) - 1) > 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_several_point_sources(O, colt, ctx, precision):
    # colt_run_params.sources: the source of each packet is an exact integer
    # choice on both sides, so in an empty box the images agree pixel for
    # pixel with the oracle's (sources at pixel centres), and in a dusty
    # outflow the 20-scattering prefixes agree packet by packet
    g = S.uniform_box((4, 4, 4), (-4e18,) * 3, (4e18,) * 3, 1e-30, 1e4)
    pos = [(-3.5e18, -3.5e18, 0.3e18), (1.5e18, -2.5e18, -0.2e18), (-2.5e18, 1.5e18, 0.1e18), (3.5e18, 3.5e18, 0.0)]
    N = 20000
    spec = S.RunSpec(n_packets=N, seed=17, spec_units=1, spec_lo=-50, spec_hi=50, spec_nbins=10,
                     cameras=S.axis_cameras(8, ("+z",)), cam_units=1, cam_lo=-50, cam_hi=50, cam_nbins=1,
                     sources=[(p, 0.0, wi) for p, wi in zip(pos, (1.0, 2.0, 5.0, 0.0))])
    rg, ro = _run_both(O, colt, ctx, g, spec, precision, per_packet=False, images=True)
    assert rg["n_escaped"] == N and np.array_equal(rg["cam_image"], ro["cam_image"])
    gd = S.sphere(24, 1e4, 1e5, v_max_kms=150.0, tau_dust=0.8)
    sp = S.RunSpec(n_packets=3000, seed=23, albedo=0.32, spec_units=1, spec_lo=-600, spec_hi=600, spec_nbins=60,
                   cameras=S.axis_cameras(0), cam_units=1, cam_lo=-600, cam_hi=600, cam_nbins=30,
                   max_scatter=PREFIX,
                   sources=[((1e17, 2e17, -3e17), 1e17, 1.0), ((-4e17, 0.0, 1e17), 0.0, 3.0),
                            ((0.0, -2e17, 2e17), 2e17, 0.5)])
    rg, ro = _run_both(O, colt, ctx, gd, sp, precision)
    full = _identity(rg, ro)
    print(f"precision {precision}: identical with frequency {full:.4f}")
    assert full >= MIN_SAME
