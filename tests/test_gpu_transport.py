"""GPU transport parity against the FP64 oracle through the C ABI.

Both sides draw every random number from Philox4x32-10 keyed by (seed, packet
id, event, block), so with the same seed a GPU packet and the oracle packet
with the same id follow the same history.  Transport is chaotic, though: a
1e-7 relative difference (the GPU's FP32 cell records) grows until a decision
flips -- the oracle against itself with n_HI perturbed by 1e-7 keeps 99.5% of
100-scattering histories and only ~15% of 8000-scattering ones.  So:
  * per-packet identity is checked on history prefixes: with max_scatter = 20
    every packet stops at its 20th scattering (or escapes/absorbs earlier) and
    both sides report status, count and the lab-frame frequency at that
    moment.  Calibration (oracle vs itself, every input perturbed by 1e-7):
    status and count agree for 100% of 20-scattering prefixes, the frequency
    within 1e-3 for 99.6%.  The GPU must reach 99% and 98%;
  * full histories are compared statistically with independent seeds:
    escape fractions within 3 sigma (two-sample binomial), per-bin chi-square
    of the spectra (p > 0.01), camera spectra against GPU batch variances;
  * conservation and integer tallies exactly; edge cases; and the full 128^3
    / 6-camera workload in the benchmark's launch configuration on packet ids
    the oracle recomputes one by one.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.special import expn

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu

PREFIX = 20
# frequency tolerance at the prefix, relative to max(1, |v|): both paths read
# FP32 cell records (1e-7) and the histories are chaotic (see above)
FTOL = {0: 1e-3, 1: 1e-3}
MIN_SAME = {0: 0.98, 1: 0.98}
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


def _identity(rg, ro, ftol):
    """(fraction identical incl. frequency, fraction with identical status and count)"""
    same = (rg["pk_status"] == ro["pk_status"]) & (rg["pk_nscat"] == ro["pk_nscat"])
    fclose = np.abs(rg["pk_freq"] - ro["pk_freq"]) <= ftol * np.maximum(1.0, np.abs(ro["pk_freq"]))
    full, disc = np.mean(same & fclose), np.mean(same)
    assert disc >= MIN_DISCRETE, disc
    return full, disc


def _conserved(r, n):
    assert r["n_emitted"] == n
    assert r["n_escaped"] + r["n_absorbed"] + r["n_capped"] == n
    assert int(r["spec"].sum()) + r["spec_under"] + r["spec_over"] == r["n_escaped"]


def cfg1_sphere():
    """32^3 static sphere, T = 10 K, tau0 = 1e5, x = 0 source, 100 bins on [-40, 40]."""
    g = S.sphere(32, 10.0, 1e5)
    spec = S.RunSpec(n_packets=1000, seed=1, T_ref=10.0, spec_units=0, spec_lo=-40, spec_hi=40, spec_nbins=100)
    return g, spec


def dusty_outflow(n=32, v=200.0, tau0=1e5):
    """A reduced-size case of the benchmark suite: T = 1e4 K, Hubble outflow, dust tau 1."""
    g = S.sphere(n, 1e4, tau0, v_max_kms=v, tau_dust=1.0)
    spec = S.RunSpec(n_packets=20000, seed=11, albedo=0.32, spec_units=1, spec_lo=-1000, spec_hi=1000,
                     spec_nbins=200, cameras=S.axis_cameras(16), cam_units=1, cam_lo=-1000, cam_hi=1000,
                     cam_nbins=200)
    return g, spec


@pytest.mark.parametrize("precision", [0, 1])
def test_cfg1_prefix_identity(O, colt, ctx, precision):
    g, spec = cfg1_sphere()
    spec.max_scatter = PREFIX
    rg, ro = _run_both(O, colt, ctx, g, spec, precision)
    _conserved(rg, 1000)
    full, same = _identity(rg, ro, FTOL[precision])
    print(f"precision {precision}: identical {same:.4f}, with frequency {full:.4f}")
    assert full >= MIN_SAME[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_dusty_outflow_prefix_identity_and_cameras(O, colt, ctx, precision):
    g, spec = dusty_outflow()
    spec.n_packets = 3000
    spec.max_scatter = PREFIX
    rg, ro = _run_both(O, colt, ctx, g, spec, precision, images=True)
    _conserved(rg, 3000)
    full, same = _identity(rg, ro, FTOL[precision])
    print(f"precision {precision}: identical {same:.4f}, with frequency {full:.4f}")
    assert full >= MIN_SAME[precision]
    # peel-off tallies of the same histories
    tol = 0.002 if precision == 0 else 0.03
    assert np.sum(np.abs(rg["cam_spec"] - ro["cam_spec"])) <= tol * np.sum(ro["cam_spec"])
    assert rg["cam_image"].sum() == pytest.approx(ro["cam_image"].sum(), rel=tol)
    img = rg["cam_image"].reshape(6, 16, 16, 200)
    assert np.allclose(img.sum(axis=(1, 2)), rg["cam_spec"], rtol=1e-9, atol=1e-300)


def _two_sample_chi2(a, b):
    a, b = a.astype(float), b.astype(float)
    na, nb = a.sum(), b.sum()
    m = (a + b) > 0
    k1, k2 = np.sqrt(nb / na), np.sqrt(na / nb)
    chi2 = np.sum((k1 * a[m] - k2 * b[m]) ** 2 / (a[m] + b[m]))
    return stats.chi2.sf(chi2, np.count_nonzero(m) - 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_cfg1_full_histories_statistics(O, colt, ctx, precision):
    # independent seeds: the GPU spectrum is a sample of the oracle's distribution
    g, spec = cfg1_sphere()
    spec.n_packets = 20000 if precision else 4000
    spec.precision = precision
    h = colt.colt_create_grid(ctx, g)
    rg = colt.colt_run(ctx, h, spec)
    colt.colt_destroy_grid(ctx, h)
    _conserved(rg, spec.n_packets)
    spec.seed = 2
    spec.n_packets = 4000
    ro = O.run(g, spec)
    assert _two_sample_chi2(rg["spec"], ro["spec"]) > 0.01
    # mean scatterings per packet agree
    mg, mo = rg["n_scat"] / rg["n_emitted"], ro["n_scat"] / ro["n_emitted"]
    assert mg == pytest.approx(mo, rel=0.1)


def test_dusty_outflow_statistics(O, colt, ctx):
    g, spec = dusty_outflow()
    spec.precision = 1
    h = colt.colt_create_grid(ctx, g)
    nb = 16
    runs = []
    for s in range(nb):
        spec.seed = 100 + s
        runs.append(colt.colt_run(ctx, h, spec))
    colt.colt_destroy_grid(ctx, h)
    spec.seed = 99
    ro = O.run(g, spec)
    N = spec.n_packets
    # escape fraction: two-sample binomial, 3 sigma
    fg = np.mean([r["n_escaped"] for r in runs]) / N
    fo = ro["n_escaped"] / N
    sig = np.sqrt(fo * (1 - fo) * (1.0 / N + 1.0 / (nb * N)))
    assert abs(fg - fo) <= 3 * sig + 1e-12
    # escape spectrum: pooled GPU runs vs oracle
    assert _two_sample_chi2(np.sum([r["spec"] for r in runs], axis=0), ro["spec"]) > 0.01
    # camera spectra (weighted, heavy-tailed): per bin the oracle value against
    # the mean of nb independent GPU batches of the same size, with the batch
    # variance; under the null z follows a t distribution with nb - 1 dof
    cam = np.stack([r["cam_spec"] for r in runs])
    mean, sd = cam.mean(axis=0), cam.std(axis=0, ddof=1)
    ok = sd > 0
    z = (ro["cam_spec"][ok] - mean[ok]) / (sd[ok] * np.sqrt(1 + 1 / nb))
    crit = stats.t.ppf(0.995, nb - 1)
    frac = np.mean(np.abs(z) > crit)
    nbins = np.count_nonzero(ok)
    assert frac <= 0.01 + 4 * np.sqrt(0.01 * 0.99 / nbins) + 2.0 / nbins, frac
    assert 0.45 < np.median(np.abs(z)) < 0.95


def test_edge_cases(O, colt, ctx):
    g = S.sphere(8, 1e4, 1e3, tau_dust=0.5)
    h = colt.colt_create_grid(ctx, g)
    # no packets
    r = colt.colt_run(ctx, h, S.RunSpec(n_packets=0, seed=1))
    assert r["n_emitted"] == 0 and r["spec"].sum() == 0
    # one packet, per-packet output
    spec = S.RunSpec(n_packets=1, seed=3, spec_units=1, spec_lo=-500, spec_hi=500, max_scatter=PREFIX)
    r = colt.colt_run(ctx, h, spec, per_packet=True)
    o = O.run(g, spec, per_packet=True)
    assert r["pk_status"][0] == o["pk_status"][0] and r["pk_nscat"][0] == o["pk_nscat"][0]
    # source outside the box: leaves at once at line centre
    out = S.RunSpec(n_packets=10, seed=3, src_pos=(1e30, 0, 0), spec_units=1, spec_lo=-5, spec_hi=5, spec_nbins=2)
    r = colt.colt_run(ctx, h, out)
    assert r["n_escaped"] == 10 and r["spec"][1] == 10 and r["n_scat"] == 0
    # narrow bins: under/overflow counted
    nb = S.RunSpec(n_packets=2000, seed=4, spec_units=1, spec_lo=-1.0, spec_hi=1.0, spec_nbins=3)
    r = colt.colt_run(ctx, h, nb)
    _conserved(r, 2000)
    assert r["spec_under"] + r["spec_over"] > 0
    # scattering cap
    cap = S.RunSpec(n_packets=500, seed=5, max_scatter=3, spec_lo=-40, spec_hi=40)
    r = colt.colt_run(ctx, h, cap, per_packet=True)
    o = O.run(g, cap, per_packet=True)
    assert r["n_capped"] > 0 and np.all(r["pk_nscat"] <= 3)
    assert np.mean(r["pk_status"] == o["pk_status"]) > 0.99
    colt.colt_destroy_grid(ctx, h)
    # a single-cell grid
    one = S.uniform_box((1, 1, 1), (-1e18, -1e18, -1e18), (1e18, 1e18, 1e18), 1e-3, 1e4, k_dust=1e-19)
    sp = S.RunSpec(n_packets=500, seed=6, spec_units=1, spec_lo=-300, spec_hi=300, max_scatter=PREFIX,
                   cameras=S.axis_cameras(2), cam_units=1, cam_lo=-300, cam_hi=300, cam_nbins=10)
    rg, ro = _run_both(O, colt, ctx, one, sp, 0, images=True)
    full, _ = _identity(rg, ro, FTOL[0])
    assert full >= 0.99
    assert np.allclose(rg["cam_spec"], ro["cam_spec"], rtol=1e-4, atol=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_grid_random_fields(O, colt, ctx, precision):
    # non-cubic cells, several 32-cell tiles along x plus a ragged tail, random
    # densities/temperatures/velocities/dust, off-centre source
    g = S.random_fields((45, 7, 13), seed=5, lo=-3e18, hi=3e18, n_range=(1e-4, 1e-2), T_range=(10, 1e5),
                        v_kms=40.0, k_dust_max=3e-19)
    g.hi = np.array([3e18, 1e18, 2e18])
    spec = S.RunSpec(n_packets=3000, seed=8, src_pos=(1.2e17, -3.3e17, 5.5e17), albedo=0.5, spec_units=1,
                     spec_lo=-600, spec_hi=600, spec_nbins=60, cameras=S.axis_cameras(0), cam_units=1,
                     cam_lo=-600, cam_hi=600, cam_nbins=60, max_scatter=PREFIX)
    rg, ro = _run_both(O, colt, ctx, g, spec, precision)
    _conserved(rg, 3000)
    full, same = _identity(rg, ro, FTOL[precision])
    assert full >= MIN_SAME[precision], (same, full)
    tol = 0.002 if precision == 0 else 0.03
    assert np.sum(np.abs(rg["cam_spec"] - ro["cam_spec"])) <= tol * np.sum(ro["cam_spec"])


def test_periodic_slab_and_absorbers(O, colt, ctx):
    g = S.slab(16, 100.0, 1e5, v_max_kms=30.0, tau_dust=0.7, nxy=3)
    spec = S.RunSpec(n_packets=3000, seed=12, albedo=0.32, T_ref=100.0, spec_lo=-60, spec_hi=60, spec_nbins=60,
                     cameras=S.axis_cameras(0), cam_units=0, cam_lo=-60, cam_hi=60, cam_nbins=60,
                     max_scatter=PREFIX)
    rg, ro = _run_both(O, colt, ctx, g, spec, 0)
    full, _ = _identity(rg, ro, FTOL[0])
    assert full >= 0.99
    # x/y cameras see nothing through a periodic slab
    assert np.all(rg["cam_spec"][:4] == 0) and rg["cam_spec"][4:].sum() > 0
    # pure absorber and perfect scatterer
    ga = S.slab(8, 1e4, 0.0, tau_dust=2.0, nxy=2)
    for A in (0.0, 1.0):
        sp = S.RunSpec(n_packets=20000, seed=13, albedo=A, spec_lo=-5, spec_hi=5)
        h = colt.colt_create_grid(ctx, ga)
        r = colt.colt_run(ctx, h, sp)
        colt.colt_destroy_grid(ctx, h)
        if A == 1.0:
            assert r["n_escaped"] == 20000
        else:
            p = expn(2, 2.0)
            assert abs(r["n_escaped"] - 20000 * p) < 4 * np.sqrt(20000 * p * (1 - p))


def test_determinism(colt, ctx):
    g, spec = dusty_outflow(n=24)
    spec.n_packets = 5000
    h = colt.colt_create_grid(ctx, g)
    r1 = colt.colt_run(ctx, h, spec, per_packet=True)
    r2 = colt.colt_run(ctx, h, spec, per_packet=True)
    colt.colt_destroy_grid(ctx, h)
    for key in ("spec", "pk_status", "pk_nscat", "pk_freq"):
        assert np.array_equal(r1[key], r2[key])
    for key in ("n_escaped", "n_absorbed", "n_scat"):
        assert r1[key] == r2[key]
    assert np.allclose(r1["cam_spec"], r2["cam_spec"], rtol=1e-12, atol=0)


def test_split_id_ranges_sum_to_the_whole(colt, ctx):
    # packets are keyed by id: two half runs (pid_offset) give the whole run's
    # integer tallies exactly (the replica/sharding contract)
    g, spec = dusty_outflow(n=16)
    spec.n_packets = 4000
    h = colt.colt_create_grid(ctx, g)
    whole = colt.colt_run(ctx, h, spec)
    a = colt.colt_run(ctx, h, S.RunSpec(**{**spec.__dict__, "n_packets": 1500}))
    b = colt.colt_run(ctx, h, S.RunSpec(**{**spec.__dict__, "n_packets": 2500, "pid_offset": 1500}))
    colt.colt_destroy_grid(ctx, h)
    assert np.array_equal(a["spec"] + b["spec"], whole["spec"])
    for key in ("n_escaped", "n_absorbed", "n_scat", "n_scat_hi"):
        assert a[key] + b[key] == whole[key]
    assert np.allclose(a["cam_spec"] + b["cam_spec"], whole["cam_spec"], rtol=1e-9, atol=1e-300)


def test_full_size_sampled_packets(O, colt, ctx):
    # the benchmark's workload (128^3 sphere, T = 1e4 K, dust tau 1, A = 0.32,
    # 6 cameras x 128^2 pixels x 200 bins), its launch configuration (a batch
    # of all nine cases in one persistent launch); the oracle recomputes
    # sampled packet ids of two cases alone, on history prefixes
    import bench
    hs, specs, grids = [], [], []
    ctxb = ctx
    N = 1 << 14
    for i, (t, v) in enumerate(bench.cases()):
        g = bench.case_grid(t, v)
        grids.append(g)
        hs.append(colt.colt_create_grid(ctxb, g))
        sp = bench.case_spec(i, N, 0, images=True)
        sp.max_scatter = PREFIX
        specs.append(sp)
    res = colt.colt_run_batch(ctxb, hs, specs, per_packet=True, images=True)
    for h in hs:
        colt.colt_destroy_grid(ctxb, h)
    # frequency criteria from the oracle's own chaos floor on these cases (all
    # inputs perturbed by 1e-7): case 4 keeps 100% within 1e-3; case 8
    # (tau0 = 1e7, outflow) 94% within 1e-3 and 97% within 1e-2
    crit = {4: (1e-3, 0.98), 8: (1e-2, 0.9)}
    for i in (4, 8):
        rg = res[i]
        _conserved(rg, N)
        img = rg["cam_image"].reshape(6, 128, 128, 200)
        assert np.allclose(img.sum(axis=(1, 2)), rg["cam_spec"], rtol=1e-9, atol=1e-300)
        for pid0 in (0, N - 150):
            sub = S.RunSpec(**{**specs[i].__dict__, "n_packets": 150, "cameras": []})
            ro = O.run(grids[i], sub, per_packet=True, pid0=pid0)
            sl = slice(pid0, pid0 + 150)
            got = {k: rg[k][sl] for k in ("pk_status", "pk_nscat", "pk_freq")}
            full, same = _identity(got, ro, crit[i][0])
            assert full >= crit[i][1], (i, pid0, same, full)


@pytest.mark.parametrize("precision", [0, 1])
def test_serving_mix_parameter_corners(O, colt, ctx, precision):
    # corners of the serving mix's parameter ranges (sphere or slab, T from 10 K
    # to 1e5 K, tau0 1e4 to 1e8, v_max +-300 km/s, dust tau 0 to 2) on small grids
    corners = [("sphere", 10.0, 1e8, 0.0, 0.0), ("slab", 1e5, 1e4, 300.0, 2.0), ("sphere", 1e5, 1e6, -300.0, 1.0),
               ("slab", 10.0, 1e6, -150.0, 0.5)]
    for geom, T, tau0, v, td in corners:
        g = S.sphere(16, T, tau0, v_max_kms=v, tau_dust=td) if geom == "sphere" else \
            S.slab(16, T, tau0, v_max_kms=v, tau_dust=td, nxy=4)
        vth = 12.85 * np.sqrt(T / 1e4)
        w = 40.0 * vth + abs(v)
        spec = S.RunSpec(n_packets=1500, seed=4100, albedo=0.32, spec_units=1, spec_lo=-w, spec_hi=w, spec_nbins=100,
                         max_scatter=PREFIX)
        rg, ro = _run_both(O, colt, ctx, g, spec, precision)
        _conserved(rg, 1500)
        full, same = _identity(rg, ro, FTOL[precision])
        print(f"{geom} T={T:g} tau0={tau0:g}: identical {same:.4f}, with frequency {full:.4f}")
        assert full >= MIN_SAME[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_natural_thermal_emission(O, colt, ctx, precision):
    # Sec. 3.1.1 emission x = x_nat + k.u_atom: in an empty box every packet
    # leaves with its emitted frequency (per packet equal to the oracle's, and the
    # emission peel-off towards each camera uses x_nat + k_c.u_atom); in the
    # dusty outflow the 20-scattering prefixes agree as with line-centre emission
    T, N = 10.0, 4000
    g = S.uniform_box((4, 4, 4), (-1e18,) * 3, (1e18,) * 3, 1e-30, T)
    spec = S.RunSpec(n_packets=N, seed=62, emission=1, T_ref=T, spec_units=0, spec_lo=-6.0, spec_hi=6.0,
                     spec_nbins=48, cameras=S.axis_cameras(0), cam_units=0, cam_lo=-6.0, cam_hi=6.0, cam_nbins=48)
    rg, ro = _run_both(O, colt, ctx, g, spec, precision)
    assert rg["n_escaped"] == N and rg["n_scat"] == 0
    # both paths read the FP32 cell records (a, 1/v_th): ~1e-7 relative
    ftol = 1e-6 if precision == 0 else 1e-5
    assert np.all(np.abs(rg["pk_freq"] - ro["pk_freq"]) <= ftol * np.maximum(1.0, np.abs(ro["pk_freq"])))
    # a frequency within rounding of a bin edge may change bins
    assert np.allclose(rg["cam_spec"].sum(axis=1), ro["cam_spec"].sum(axis=1), rtol=1e-6)
    assert np.sum(np.abs(rg["cam_spec"] - ro["cam_spec"])) <= 0.01 * np.sum(ro["cam_spec"])
    g, spec = dusty_outflow()
    spec.n_packets, spec.max_scatter, spec.emission = 3000, PREFIX, 1
    rg, ro = _run_both(O, colt, ctx, g, spec, precision, images=True)
    full, same = _identity(rg, ro, FTOL[precision])
    print(f"precision {precision}: identical {same:.4f}, with frequency {full:.4f}")
    assert full >= MIN_SAME[precision]
