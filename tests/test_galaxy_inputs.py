"""Pins of the idealized first-galaxy models of Sec. 5.1 (inputs; no GPU).

Closed forms and printed values: n_H,IGM ~ 2e-4 ((1+z)/10)^3 cm^-3; chi = 560
for M_H,tot = 1e7 Msun, r_core = 10 pc, z = 9 (Eq. chi); Eq. MHtot against a
quadrature of the profile; Eq. nH0's large-mass expansion against the exact
root to 1e-9 above 1e6 Msun (the paper's claim); the edge radii 1.09, 2.35,
5.05 and 10.88 kpc the radial-profile figure prints for the 5- to 8-models; the
Stromgren radius 15 pc of Eq. stromgren; and the generated octrees: hydrogen
mass, ionized regions, wind law and refinement criteria."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_1409_4480_gb300 import synth as S

KPC = 1e3 * S.PC_CM


def test_igm_density_and_chi():
    assert S.n_h_igm(9.0) == pytest.approx(2e-4, rel=0.1)
    assert S.n_h_igm(19.0) / S.n_h_igm(9.0) == pytest.approx(8.0, rel=1e-12)
    assert S.galaxy_chi(1e7, 10 * S.PC_CM, 9.0) == pytest.approx(560.0, rel=0.01)
    assert S.galaxy_chi(8e7, 10 * S.PC_CM, 9.0) / S.galaxy_chi(1e7, 10 * S.PC_CM, 9.0) == pytest.approx(2.0)
    assert S.galaxy_chi(1e7, 20 * S.PC_CM, 19.0) / S.galaxy_chi(1e7, 10 * S.PC_CM, 9.0) == pytest.approx(0.25)


@pytest.mark.parametrize("M", [1e5, 1e6, 1e7, 1e8])
def test_core_density_normalises_the_mass(M):
    z, rc = 9.0, 10 * S.PC_CM
    n0, ni = S.galaxy_core_density(M, rc, z), S.n_h_igm(z)
    re = rc * math.sqrt(n0 / ni)
    prof = lambda r: n0 if r <= rc else n0 * (rc / r) ** 2
    m_quad = 4 * math.pi * S.M_H_G * (integrate.quad(lambda r: prof(r) * r * r, 0, rc)[0]
                                      + integrate.quad(lambda r: prof(r) * r * r, rc, re)[0])
    assert m_quad == pytest.approx(M * S.MSUN_G, rel=1e-10)
    # Eq. MHtot's closed form
    assert 4 * math.pi * S.M_H_G * n0 * rc ** 3 * (math.sqrt(n0 / ni) - 2 / 3) == pytest.approx(M * S.MSUN_G, rel=1e-12)
    # Eq. nH0: n0 ~ n_IGM (chi^2 + 4 chi / 9 + 4/27), "better than 1e-9 for
    # masses larger than 1e6 Msun" (the next term is O(chi^-3): 2e-9 at 1e6 itself)
    chi = S.galaxy_chi(M, rc, z)
    approx = ni * (chi * chi + 4 * chi / 9 + 4 / 27)
    tol = {1e5: 1e-7, 1e6: 3e-9}.get(M, 1e-9)
    assert abs(approx / n0 - 1) < tol


def test_edge_radii_printed():
    for M, r_kpc in ((1e5, 1.09), (1e6, 2.35), (1e7, 5.05), (1e8, 10.88)):
        n0 = S.galaxy_core_density(M, 10 * S.PC_CM, 10.0)
        r_edge = 10 * S.PC_CM * math.sqrt(n0 / S.n_h_igm(10.0))
        assert r_edge / KPC == pytest.approx(r_kpc, rel=0.01)


def test_stromgren_radius_printed():
    # Eq. stromgren with alpha_B = 2.5e-13 T4^-3/4: 15 pc at T4 = 1, Ndot = 1e51 s^-1, n = 100 cm^-3
    rs = (3 / (4 * math.pi) * 1e51 / (100.0 ** 2 * 2.5e-13)) ** (1 / 3)
    assert rs / S.PC_CM == pytest.approx(15.0, rel=0.03)


def _small(model, M):
    return S.galaxy(model, M, n_jeans=8, n_geo=8, n_cone=32)


def test_galaxy_grid_mass_and_ionisation():
    g = S.galaxy("SE", 1e6)
    m = g.meta
    c, s = S.leaf_geometry(g.lo, g.hi, g.leaf_level, g.leaf_ijk)
    r = np.linalg.norm(c, axis=1)
    vol = np.prod(s, axis=1)
    nhi = g.n_HI.astype(np.float64)
    # early: the Stromgren sphere (R_S = r_core) holds no neutral hydrogen
    assert np.all(nhi[r < m["r_core"]] == 0)
    shell = (r >= m["r_core"]) & (r < m["r_edge"])
    m_shell = np.sum(nhi[shell] * vol[shell]) * S.M_H_G
    exact = 4 * math.pi * S.M_H_G * m["n_h0"] * m["r_core"] ** 3 * (math.sqrt(m["n_h0"] / m["n_h_igm"]) - 1)
    assert m_shell == pytest.approx(exact, rel=0.03)
    assert np.allclose(nhi[r >= m["r_edge"]], m["n_h_igm"], rtol=1e-6)
    # refinement: neutral leaves are at most lambda_J / 64 and r_edge / 64 on the edge sphere
    neutral = nhi > 0
    lam = S.jeans_length(1e4, nhi[neutral])
    assert np.all(s[neutral, 0] * 64 <= lam * (1 + 1e-12))
    on_edge = np.abs(r - m["r_edge"]) < 0.5 * np.linalg.norm(s, axis=1)
    assert np.all(s[on_edge, 0] * 64 <= m["r_edge"] * (1 + 1e-12))


def test_late_cone_and_wind_law():
    g = _small("WL", 1e6)
    m = g.meta
    c, s = S.leaf_geometry(g.lo, g.hi, g.leaf_level, g.leaf_ijk)
    r = np.linalg.norm(c, axis=1)
    in_cone = (np.abs(c[:, 2]) > math.cos(math.radians(30)) * r) & (r < m["r_edge"])
    assert np.all(g.n_HI[in_cone] == 0)
    assert np.all(g.n_HI[~in_cone & (r > m["r_core"])] > 0)
    v = np.stack([g.vx, g.vy, g.vz], axis=1).astype(np.float64)
    sel = r > 2 * m["r_star"]
    speed = np.linalg.norm(v[sel], axis=1)
    expect = 10.0 * np.sqrt(1 - m["r_star"] / r[sel])
    assert np.allclose(speed, expect, rtol=1e-5)
    # radial
    cosang = np.sum(v[sel] * c[sel], axis=1) / (speed * r[sel])
    assert np.all(cosang > 1 - 1e-5)
