"""Recoil in cold, thick gas (App. "Thermal effects on Ly-alpha spectra"),
oracle only (no GPU).

Eq. x_f moves a photon by g (k_i.k_f - 1) per scattering, on average -g (the
phase function has <mu> = 0), i.e. to the red (x < 0, Delta v > 0), by
g = 2.536e-4 T4^-1/2 -- a shift that matters only where the Lorentzian part
of the redistribution is small, in cold gas.  Without recoil a static slab's
spectrum is symmetric; with it, a 10 K slab of tau_0 = 1e7 is strongly red and
a 1e4 K one nearly symmetric."""
import numpy as np

from paper_1409_4480_gb300 import synth as S


def _asym(spec):
    s = spec.astype(float)
    h = len(s) // 2
    return (s[h:].sum() - s[:h].sum()) / s.sum()


def test_recoil_reddens_cold_thick_slabs(O):
    out = {}
    for T, recoil in ((10.0, True), (10.0, False), (1e3, True)):
        spec = S.RunSpec(n_packets=1500, seed=150, recoil=recoil, T_ref=T, spec_units=1, spec_lo=-100.0,
                         spec_hi=100.0, spec_nbins=40)
        r = O.run(S.slab(16, T, 1e7, nxy=2), spec)
        assert r["n_escaped"] == 1500
        out[(T, recoil)] = _asym(r["spec"])
    noise = 1.0 / np.sqrt(1500)
    assert abs(out[(10.0, False)]) < 4 * noise            # symmetric without recoil
    assert out[(10.0, True)] > 0.3                         # red excess with recoil at 10 K
    assert out[(10.0, True)] > out[(1e3, True)] + 4 * noise
