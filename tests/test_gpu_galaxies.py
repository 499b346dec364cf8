"""The idealized first-galaxy models of Sec. 5.1 on the GPU.

  * parity: 20-scattering history prefixes against the oracle on coarse
    octrees of an early static and a late wind model, with the Jeans
    core-skipping estimate and with the cell + non-local one;
  * the paper's flux table for the M_H,tot = 1e6 Msun early wind and late
    models, on coarser octrees than the paper's, 3000 packets, cell + non-local
    core-skipping: late models are brighter face-on (z) than edge-on (xy),
    within 25 per cent of the printed F/F_Omega; winds are red (F_r/F_b > 1),
    the early wind near the printed 5.72, the late one lower and ordered
    z < Omega < xy, within 25 per cent of the printed values; the static model
    is symmetric.  The 25 per cent is the model freedom the paper leaves (cone
    and IGM discretisation, resolution, statistics).  A few histories run to
    ~1e7 scatterings alone on one lane; they are capped at 3e6 (under 1 per
    cent of the packets, checked) so that the test takes seconds.  The full
    16-model suite at the paper's refinement is `bench.py --workload galaxies`."""
import numpy as np
import pytest

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu

# paper's flux table: F/F_Omega along z and xy, F_r/F_b along z, Omega, xy
PAPER_F = {("SL", 6): (1.60, 0.72), ("WL", 6): (1.80, 0.74)}
PAPER_RB = {("WL", 6): (2.96, 3.49, 4.58), ("WE", 6): (None, 5.72, None)}
MODELS = [("WE", 6), ("SL", 6), ("WL", 6)]
N_FLUX, CAP = 3000, 3_000_000


@pytest.fixture(scope="module")
def ctx(colt):
    c = colt.colt_init(0)
    yield c
    colt.colt_finalize(c)


def _spec(n, seed, core_skip=1, **kw):
    return S.RunSpec(n_packets=n, seed=seed, core_skip=core_skip, albedo=0.0, spec_units=1, spec_lo=-3000.0,
                     spec_hi=3000.0, spec_nbins=300, cameras=S.axis_cameras(0), cam_units=1, cam_lo=-3000.0,
                     cam_hi=3000.0, cam_nbins=300, **kw)


@pytest.mark.parametrize("model,M", [("SE", 1e5), ("WL", 1e6)])
def test_galaxy_prefix_identity(O, colt, ctx, model, M):
    g = S.galaxy(model, M, n_jeans=8, n_geo=8, n_cone=32)
    for precision, skip in ((0, 2), (1, 2), (1, 1)):
        spec = _spec(3000, 170, core_skip=skip, max_scatter=20, precision=precision)
        h = colt.colt_create_grid(ctx, g)
        try:
            rg = colt.colt_run(ctx, h, spec, per_packet=True)
        finally:
            colt.colt_destroy_grid(ctx, h)
        ro = O.run(g, spec, per_packet=True)
        same = (rg["pk_status"] == ro["pk_status"]) & (rg["pk_nscat"] == ro["pk_nscat"])
        close = np.abs(rg["pk_freq"] - ro["pk_freq"]) <= 1e-3 * np.maximum(1.0, np.abs(ro["pk_freq"]))
        print(f"{model}{int(np.log10(M))} precision {precision} core_skip {skip}: identical {same.mean():.4f}, "
              f"with frequency {(same & close).mean():.4f}")
        assert same.mean() >= 0.99 and (same & close).mean() >= 0.98


def _observables(r):
    cs = np.asarray(r["cam_spec"], np.float64)            # +x -x +y -y +z -z
    esc = float(np.sum(r["spec"]))
    h = cs.shape[1] // 2
    rb = lambda s: s[h:].sum() / s[:h].sum()
    sp = np.asarray(r["spec"], np.float64)
    return dict(Fz=cs[4:6].sum(axis=1).mean() / esc, Fxy=cs[0:4].sum(axis=1).mean() / esc,
                rb_z=rb(cs[4:6].sum(axis=0)), rb_xy=rb(cs[0:4].sum(axis=0)), rb_O=rb(sp))


def test_flux_table_trends(colt, ctx):
    out = {}
    for m, lg in MODELS:
        g = S.galaxy(m, 10.0 ** lg, n_jeans=16, n_geo=16, n_cone=64)
        h = colt.colt_create_grid(ctx, g)
        try:
            r = colt.colt_run(ctx, h, _spec(N_FLUX, 180 + lg, max_scatter=CAP))
        finally:
            colt.colt_destroy_grid(ctx, h)
        assert r["n_escaped"] + r["n_capped"] == N_FLUX and r["n_capped"] < 0.01 * N_FLUX
        out[(m, lg)] = o = _observables(r)
        print(m, lg, {k: round(float(v), 3) for k, v in o.items()}, f"{r['kernel_ms'] / 1e3:.1f} s")
    for (m, lg), (fz, fxy) in PAPER_F.items():
        o = out[(m, lg)]
        assert o["Fz"] > 1.2 and o["Fxy"] < 0.95
        assert o["Fz"] == pytest.approx(fz, rel=0.25) and o["Fxy"] == pytest.approx(fxy, rel=0.25)
    for (m, lg), vals in PAPER_RB.items():
        o = out[(m, lg)]
        for key, ref in zip(("rb_z", "rb_O", "rb_xy"), vals):
            if ref is not None:
                assert o[key] == pytest.approx(ref, rel=0.25)
    wl = out[("WL", 6)]
    assert 1.0 < wl["rb_z"] < wl["rb_O"] < wl["rb_xy"]
    assert out[("SL", 6)]["rb_O"] == pytest.approx(1.0, abs=0.1)
    assert out[("WE", 6)]["Fz"] == pytest.approx(out[("WE", 6)]["Fxy"], rel=0.1)
    assert out[("WE", 6)]["rb_O"] > wl["rb_O"]
