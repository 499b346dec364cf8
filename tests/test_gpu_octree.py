"""GPU parity on octree grids against the FP64 oracle, through the C ABI.

  * per-leaf records and the octree a tau_NL (Eq. atauNL) equal the oracle's;
  * pure absorber on a mixed-level octree: every camera's emission peel-off is
    exp(-tau) of the axis ray (Sec. 6.1), the same on both sides;
  * history prefixes (max_scatter = 20) on a refined sphere and on a synthetic
    halo (five levels, velocities, two temperatures, six cameras) agree packet
    by packet, as on Cartesian grids (the chaos calibration there applies);
  * full histories agree statistically (escape fraction, spectrum chi-square);
  * the octree of a 2^L Cartesian cube gives the Cartesian results;
  * an octree and a Cartesian request served together; invalid trees.
"""
import numpy as np
import pytest
from scipy import stats

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu

R = S.PC_CM
PREFIX = 20
FTOL = 1e-3
MIN_SAME = 0.98
MIN_DISCRETE = 0.99


@pytest.fixture(scope="module")
def ctx(colt):
    c = colt.colt_init(0)
    yield c
    colt.colt_finalize(c)


def _run(colt, ctx, g, spec, per_packet=True, images=False):
    h = colt.colt_create_grid(ctx, g, f_nl=spec.f_nl)
    try:
        return colt.colt_run(ctx, h, spec, per_packet=per_packet, images=images)
    finally:
        colt.colt_destroy_grid(ctx, h)


def _identity(rg, ro):
    same = (rg["pk_status"] == ro["pk_status"]) & (rg["pk_nscat"] == ro["pk_nscat"])
    fclose = np.abs(rg["pk_freq"] - ro["pk_freq"]) <= FTOL * np.maximum(1.0, np.abs(ro["pk_freq"]))
    return np.mean(same & fclose), np.mean(same)


def _random_octree(seed, min_level=1, max_level=5, p=0.45):
    rng = np.random.default_rng(seed)
    lo, hi = np.array([-R] * 3), np.array([R] * 3)
    lv, ijk = S.octree_refine(lo, hi, lambda c, s, L: rng.uniform(size=len(c)) < p, min_level, max_level)
    return lo, hi, lv, ijk


def small_halo():
    return S.halo(seed=13, min_level=5, max_level=10, cone_level=7, leaf_mass_frac=2e-4)


def test_octree_records_and_atau_nl(O, colt, ctx):
    for g in (S.octree_sphere(1e4, 1e5, v_max_kms=50.0, tau_dust=0.5, min_level=2, max_level=5), small_halo()):
        h = colt.colt_create_grid(ctx, g, f_nl=0.5)
        rec = colt.colt_read_cells(ctx, h, g.n_cells).astype(np.float64)
        colt.colt_destroy_grid(ctx, h)
        T = g.T.astype(np.float64)
        vth = np.array([O.vth_kms(t) for t in T])
        exp = np.stack([g.n_HI * np.array([O.sigma0(t) for t in T]), [O.damping_a(t) for t in T],
                        g.k_dust.astype(np.float64), 1.0 / vth, g.vx / vth, g.vy / vth, g.vz / vth], axis=1)
        assert np.allclose(rec[:, :7], exp, rtol=2e-7, atol=0)
        atnl = O.atau_nl(g, 0.5)
        assert np.count_nonzero(atnl) > 0
        assert np.allclose(rec[:, 7], atnl, rtol=2e-6, atol=1e-30)


@pytest.mark.parametrize("precision,rel", [(0, 1e-9), (1, 2e-5)])
def test_octree_peel_attenuation(O, colt, ctx, precision, rel):
    lo, hi, lv, ijk = _random_octree(6)
    kd = np.random.default_rng(7).uniform(0.2, 3.0, len(lv)) / R
    g = S.octree_grid(lo, hi, lv, ijk, dict(n_HI=np.zeros(len(lv)), T=np.full(len(lv), 1e4), k_dust=kd))
    N = 256
    spec = S.RunSpec(n_packets=N, seed=8, albedo=0.0, spec_lo=-5, spec_hi=5,
                     src_pos=(0.1234 * R, -0.2345 * R, 0.3456 * R), cameras=S.axis_cameras(0),
                     cam_units=0, cam_lo=-5, cam_hi=5, cam_nbins=10, precision=precision)
    rg = _run(colt, ctx, g, spec, per_packet=False)
    ro = O.run(g, spec)
    assert np.allclose(rg["cam_spec"].sum(axis=1), ro["cam_total"], rtol=rel, atol=0)
    assert rg["n_absorbed"] + rg["n_escaped"] == N


@pytest.mark.parametrize("precision", [0, 1])
def test_octree_sphere_prefix_identity(O, colt, ctx, precision):
    g = S.octree_sphere(1e4, 1e5, v_max_kms=100.0, tau_dust=1.0, min_level=3, max_level=6)
    spec = S.RunSpec(n_packets=3000, seed=17, albedo=0.32, spec_units=1, spec_lo=-800, spec_hi=800, spec_nbins=160,
                     cameras=S.axis_cameras(8), cam_lo=-800, cam_hi=800, cam_nbins=80, max_scatter=PREFIX,
                     src_pos=(0.01 * R, -0.02 * R, 0.015 * R), precision=precision)
    rg = _run(colt, ctx, g, spec, images=True)
    ro = O.run(g, spec, per_packet=True, images=True)
    full, disc = _identity(rg, ro)
    print(f"precision {precision}: identical {disc:.4f}, with frequency {full:.4f}")
    assert disc >= MIN_DISCRETE and full >= MIN_SAME
    tol = 0.002 if precision == 0 else 0.03
    assert np.sum(np.abs(rg["cam_spec"] - ro["cam_spec"])) <= tol * np.sum(ro["cam_spec"])
    assert rg["cam_image"].sum() == pytest.approx(ro["cam_image"].sum(), rel=tol)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("src_pos,src_sigma", [((0.0, 0.0, 0.0), 100.0 * R),          # central Gaussian
                                               ((0.0, 0.0, 300.0 * R), 0.0),        # in the ionised cone
                                               ((200.0 * R, -100.0 * R, 350.0 * R), 0.0)])
def test_halo_prefix_identity(O, colt, ctx, precision, src_pos, src_sigma):
    g = small_halo()
    assert len(np.unique(g.leaf_level)) >= 4
    spec = S.RunSpec(n_packets=2000, seed=23, albedo=0.32, spec_units=1, spec_lo=-1000, spec_hi=1000,
                     spec_nbins=200, cameras=S.axis_cameras(0), cam_lo=-1000, cam_hi=1000, cam_nbins=100,
                     src_pos=src_pos, src_sigma=src_sigma, max_scatter=PREFIX, precision=precision)
    rg = _run(colt, ctx, g, spec)
    ro = O.run(g, spec, per_packet=True)
    full, disc = _identity(rg, ro)
    print(f"precision {precision}: identical {disc:.4f}, with frequency {full:.4f}")
    # The clumpy halo is far more chaotic than the spheres: the oracle against
    # itself with the source moved by a relative 1e-9 keeps 99.65% of the
    # 20-scattering frequencies within 1e-3 (1e-7: 85.7%, off-centre source).
    # FP32 transport rounds at ~6e-8 per operation, so it is held to 95%.
    assert disc >= MIN_DISCRETE and full >= (MIN_SAME if precision == 0 else 0.95)
    tol = 0.002 if precision == 0 else 0.03
    assert np.sum(np.abs(rg["cam_spec"] - ro["cam_spec"])) <= tol * np.sum(ro["cam_spec"])


def test_octree_full_histories_statistics(O, colt, ctx):
    g = S.octree_sphere(1e4, 1e5, v_max_kms=-150.0, tau_dust=1.0, min_level=3, max_level=5)
    spec = S.RunSpec(n_packets=6000, seed=31, albedo=0.32, spec_units=1, spec_lo=-800, spec_hi=800, spec_nbins=40)
    rg = _run(colt, ctx, g, spec, per_packet=False)
    spec.seed = 32
    ro = O.run(g, spec)
    n = spec.n_packets
    f1, f2 = rg["n_escaped"] / n, ro["n_escaped"] / n
    p = 0.5 * (f1 + f2)
    assert abs(f1 - f2) <= 3.5 * np.sqrt(p * (1 - p) * 2 / n) + 1e-12
    a, b = rg["spec"].astype(float), ro["spec"].astype(float)
    m = (a + b) > 0
    ka, kb = np.sqrt(b.sum() / a.sum()), np.sqrt(a.sum() / b.sum())
    chi2 = np.sum((ka * a[m] - kb * b[m]) ** 2 / (a[m] + b[m]))
    assert stats.chi2.sf(chi2, np.count_nonzero(m) - 1) > 0.01


@pytest.mark.parametrize("precision", [0, 1])
def test_octree_of_cartesian_cube(colt, ctx, precision):
    gc = S.sphere(16, 1e4, 1e5, v_max_kms=80.0, tau_dust=0.7)
    go = S.octree_from_cartesian(gc, seed=5)
    spec = S.RunSpec(n_packets=2000, seed=41, albedo=0.32, spec_units=1, spec_lo=-400, spec_hi=400, spec_nbins=80,
                     cameras=S.axis_cameras(0), cam_lo=-400, cam_hi=400, cam_nbins=40, max_scatter=PREFIX,
                     src_pos=(0.13 * R, -0.21 * R, 0.05 * R), precision=precision)
    rc = _run(colt, ctx, gc, spec)
    ro = _run(colt, ctx, go, spec)
    full, disc = _identity(ro, rc)
    assert disc >= 0.995 and full >= 0.99


def test_octree_single_leaf_and_vertex_source(O, colt, ctx):
    # the root as the only leaf; then a source exactly on a vertex shared by many leaves
    g1 = S.octree_grid([-R] * 3, [R] * 3, np.zeros(1, np.uint8), np.zeros((1, 3), np.uint32),
                       dict(n_HI=[S.sigma0_recipe(1e4) ** -1 * 1e3 / R], T=[1e4]))
    spec = S.RunSpec(n_packets=500, seed=3, spec_units=1, spec_lo=-300, spec_hi=300, spec_nbins=30,
                     cameras=S.axis_cameras(0), cam_lo=-300, cam_hi=300, cam_nbins=30, max_scatter=PREFIX)
    rg = _run(colt, ctx, g1, spec)
    ro = O.run(g1, spec, per_packet=True)
    assert _identity(rg, ro)[1] >= MIN_DISCRETE
    g2 = S.octree_sphere(1e4, 1e4, min_level=2, max_level=4)
    spec.src_pos = (0.0, 0.0, 0.0)
    rg = _run(colt, ctx, g2, spec)
    ro = O.run(g2, spec, per_packet=True)
    assert _identity(rg, ro)[1] >= MIN_DISCRETE


def test_octree_and_cartesian_served_together(colt, ctx):
    go = S.octree_sphere(1e4, 1e5, min_level=3, max_level=5)
    gc = S.sphere(16, 1e4, 1e5)
    ho, hc = colt.colt_create_grid(ctx, go), colt.colt_create_grid(ctx, gc)
    spec = S.RunSpec(n_packets=3000, seed=5, spec_units=1, spec_lo=-500, spec_hi=500, spec_nbins=50)
    try:
        want = [colt.colt_run(ctx, h, spec) for h in (ho, hc)]
        rids = [colt.colt_submit(ctx, h, spec) for h in (ho, hc, ho)]
        for rid in rids:
            colt.colt_wait(ctx, rid, -1.0)
        got = [colt.colt_read_result(ctx, rid, spec) for rid in rids]
        for rid in rids:
            colt.colt_release(ctx, rid)
        for gr, wr in zip(got, [want[0], want[1], want[0]]):
            assert np.array_equal(gr["spec"], wr["spec"])
            assert gr["n_scat"] == wr["n_scat"]
        with pytest.raises(colt.ColtError):
            colt.colt_run_batch(ctx, [ho, hc], [spec, spec])
    finally:
        colt.colt_destroy_grid(ctx, ho)
        colt.colt_destroy_grid(ctx, hc)


def test_invalid_octrees_rejected(colt, ctx):
    lo, hi, lv, ijk = _random_octree(2, max_level=3)
    f = dict(n_HI=np.ones(len(lv)), T=np.full(len(lv), 1e4))
    bad = [
        (lv[:-1], ijk[:-1], {k: v[:-1] for k, v in f.items()}),                   # a hole
        (np.r_[lv, lv[:1]], np.r_[ijk, ijk[:1]], {k: np.r_[v, v[:1]] for k, v in f.items()}),  # a duplicate
        (np.r_[lv, [0]].astype(np.uint8), np.r_[ijk, [[0, 0, 0]]].astype(np.uint32),
         {k: np.r_[v, v[:1]] for k, v in f.items()}),                              # overlaps everything
        (lv, np.where(ijk == 0, 1 << 20, ijk).astype(np.uint32), f),               # coordinate outside its level
    ]
    for blv, bijk, bf in bad:
        with pytest.raises(colt.ColtError) as e:
            colt.colt_create_grid(ctx, S.octree_grid(lo, hi, blv, bijk, bf))
        assert e.value.code == colt.COLT_EINVAL


def small_cosmo():
    return S.cosmo_box(n_fft=32, min_level=4, max_level=8, leaf_mass_frac=2e-4)


@pytest.mark.parametrize("precision", [0, 1])
def test_cosmo_box_prefix_identity(O, colt, ctx, precision):
    # Sources at the highest peaks of the FFT grid lie on octree split planes
    # (both sides apply the same tie rule).  This medium is the most chaotic:
    # the oracle against itself with every input field moved by one FP32 ulp
    # (the resolution of the GPU's cell records) keeps 88.8-90% of the
    # 20-scattering frequencies within 1e-3, but 99.4-99.6% of 10-scattering
    # ones, so the prefix here is 10 scatterings.
    g, src = small_cosmo()
    assert len(np.unique(g.leaf_level)) >= 3
    for j in (0, 3):
        spec = S.RunSpec(n_packets=2000, seed=51 + j, albedo=0.32, spec_units=1, spec_lo=-500, spec_hi=500,
                         spec_nbins=100, cameras=S.axis_cameras(0, ("+x", "+y", "+z")), cam_lo=-500, cam_hi=500,
                         cam_nbins=50, src_pos=src[j], max_scatter=10, precision=precision)
        rg = _run(colt, ctx, g, spec)
        ro = O.run(g, spec, per_packet=True)
        full, disc = _identity(rg, ro)
        print(f"source {j} precision {precision}: identical {disc:.4f}, with frequency {full:.4f}")
        assert disc >= MIN_DISCRETE and full >= (MIN_SAME if precision == 0 else 0.95)
