"""The idealized first-galaxy models of Sec. 5.1 on the GPU: 20-scattering
history prefixes against the oracle on coarse octrees of an early static and
a late wind model, with the Jeans core-skipping estimate and with the cell +
non-local one.  (The paper's flux table is compared by `bench.py --workload
galaxies`, which runs the 16 models at the paper's refinement: their
histories reach 1e7-1e8 scatterings, minutes of one lane's latency, too long
for a test.)"""
import numpy as np
import pytest

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu


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
