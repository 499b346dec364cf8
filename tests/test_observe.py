"""Pins of the observables of Sec. 6.1 (host post-processing, no GPU).

  * luminosity distance: the Einstein-de Sitter closed form and the low-z
    expansion;
  * Eq. SB's unit factor L / [4 pi N (1+z)^4 206265^2 l_pix^2] equals
    L / (4 pi N d_L^2 Omega_pix) with d_L = (1+z)^2 d_A, Omega_pix = (l_pix/d_A)^2
    (the paper's footnote);
  * flux conservation: in an empty box every packet's emission peel-off has
    weight 1, so the surface brightness summed over the pixels' solid angles,
    and the flux density integrated over observed wavelength, are L/(4 pi d_L^2);
  * half-light radius and radial profile of a Gaussian map;
  * Eq. tauGP: the printed tau_0(z) and R_alpha, and the wing integral against
    its closed-form antiderivative (sympy) where R_alpha^2 x^6 is negligible."""
import math

import numpy as np
import pytest

from paper_1409_4480_gb300 import observe as ob
from paper_1409_4480_gb300 import synth as S


def test_luminosity_distance_closed_forms():
    eds = ob.Cosmology(H0_kms_mpc=70.0, omega_m=1.0)
    h0 = 70.0 * 1e5 / ob.MPC_CM
    for z in (0.5, 3.0, 9.0):
        exact = 2.0 * ob.C_CMS / h0 * (1.0 + z) * (1.0 - 1.0 / math.sqrt(1.0 + z))
        assert ob.luminosity_distance(z, eds) == pytest.approx(exact, rel=1e-9)
    # low z: c z / H0 (1 + (1 - q0) z / 2), q0 = Om/2 - OL
    c = ob.PLANCK13
    z = 1e-3
    q0 = c.omega_m / 2 - c.omega_l
    h0 = c.H0_kms_mpc * 1e5 / ob.MPC_CM
    assert ob.luminosity_distance(z, c) == pytest.approx(ob.C_CMS * z / h0 * (1 + (1 - q0) * z / 2), rel=1e-6)


def test_sb_factor_is_the_solid_angle_form():
    L, N, z, l_pix = 1e42, 10 ** 6, 9.0, 3e20
    dl, da = ob.luminosity_distance(z), ob.angular_diameter_distance(z)
    omega_arcsec2 = (l_pix / da) ** 2 * ob.ARCSEC_PER_RAD ** 2
    assert ob.sb_factor(L, N, z, l_pix) == pytest.approx(L / (4 * math.pi * N * dl * dl * omega_arcsec2), rel=1e-12)
    assert ob.ARCSEC_PER_RAD == pytest.approx(206265, rel=1e-5)


def test_flux_conservation_through_the_units(O):
    g = S.uniform_box((4, 4, 4), (-1e20,) * 3, (1e20,) * 3, 0.0, 1e4)
    N, L, z = 20000, 3e42, 9.0
    spec = S.RunSpec(n_packets=N, seed=160, spec_units=1, spec_lo=-100, spec_hi=100, spec_nbins=4,
                     cameras=S.axis_cameras(16, ("+z",)), cam_units=1, cam_lo=-100, cam_hi=100, cam_nbins=4)
    r = O.run(g, spec, images=True)
    fov = 1e20
    img = r["cam_image"].reshape(16, 16, 4)
    sb = ob.surface_brightness(img, L, N, z, fov)
    omega = (ob.pixel_size(fov, 16) / ob.angular_diameter_distance(z)) ** 2 * ob.ARCSEC_PER_RAD ** 2
    F = L / (4 * math.pi * ob.luminosity_distance(z) ** 2)
    assert sb.sum() * omega == pytest.approx(F, rel=1e-9)
    fl = ob.flux_density(r["cam_spec"][0], L, N, z, -100, 100)
    dl = np.diff(ob.observed_wavelength(ob.velocity_edges(-100, 100, 4), z))
    assert np.sum(fl * dl) == pytest.approx(F, rel=1e-9)


def test_half_light_radius_and_profile_of_a_gaussian():
    npix, fov, sig = 256, 1.0, 0.1
    c = (np.arange(npix) + 0.5) * (2 * fov / npix) - fov
    r2 = c[None, :] ** 2 + c[:, None] ** 2
    m = np.exp(-0.5 * r2 / sig ** 2)
    assert ob.half_light_radius(m, fov) == pytest.approx(sig * math.sqrt(2 * math.log(2)), rel=0.01)
    rc, prof = ob.radial_profile(m, fov, nbins=20)
    sel = rc < 3 * sig
    assert np.allclose(prof[sel], np.exp(-0.5 * rc[sel] ** 2 / sig ** 2), rtol=0.05, atol=0.01)


def test_gunn_peterson_constants():
    assert ob.tau_gp_line_centre(9.0) == pytest.approx(7e5, rel=1e-12)
    assert ob.r_alpha() == pytest.approx(2e-8, rel=0.02)


def test_wing_integral_closed_form():
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x", positive=True)
    F = sp.lambdify(x, sp.integrate(x ** sp.Rational(9, 2) / (1 - x) ** 2, x), "mpmath")
    for x0, x1 in ((0.5, 0.9), (0.95, 0.999), (0.2, 0.99)):
        exact = float((F(x1) - F(x0)).real)
        assert ob._wing_integral(x0, x1, ob.r_alpha()) == pytest.approx(exact, rel=1e-7)


def test_igm_transmission_rises_to_the_red():
    z = 9.0
    t = ob.igm_transmission(0.0, 2000.0, 20, z_em=z, z_i=z - 0.05, z_rei=6.0)
    assert np.all(np.diff(t) > 0)
    assert 0.0 <= t[0] < t[-1] <= 1.0
    # a larger ionised bubble (z_i further below z_em) transmits more
    t2 = ob.igm_transmission(0.0, 2000.0, 20, z_em=z, z_i=z - 0.2, z_rei=6.0)
    assert np.all(t2 > t)
