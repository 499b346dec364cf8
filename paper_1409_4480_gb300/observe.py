"""Observables from the peel-off tallies (Sec. 6.1): surface brightness and
flux density in physical units, radial profiles and half-light radii, and the
IGM red damping wing (Eq. tauGP).

Host post-processing of what the GPU solve returns (camera image cubes and
camera spectra, both sums of W exp(-tau_esc) over the peel-off events, Eq. SB);
nothing here runs per packet.

Units: cm, s, erg; camera spectra binned in Doppler velocity Delta v (km/s,
red = positive, Delta v = c Delta lambda / lambda).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import integrate

C_CMS = 2.99792458e10
C_KMS = 2.99792458e5
LAMBDA_LYA_CM = 1215.67e-8          # rest wavelength
A_LYA = 6.265e8                     # Einstein coefficient (natural width Lambda), s^-1
ARCSEC_PER_RAD = 180.0 / math.pi * 3600.0   # ~206265 (Sec. 6.1 footnote)
MPC_CM = 3.0856775814913673e24


@dataclass(frozen=True)
class Cosmology:
    """Flat Lambda-CDM (Sec. 5.1 takes Planck 2013 parameters)."""
    H0_kms_mpc: float = 67.8
    omega_m: float = 0.307

    @property
    def omega_l(self) -> float:
        return 1.0 - self.omega_m

    def hubble(self, z):
        """H(z) in s^-1."""
        h0 = self.H0_kms_mpc * 1e5 / MPC_CM
        return h0 * np.sqrt(self.omega_m * (1.0 + z) ** 3 + self.omega_l)


PLANCK13 = Cosmology()


def comoving_distance(z: float, cosmo: Cosmology = PLANCK13) -> float:
    """int_0^z c dz' / H(z') (cm)."""
    val, _ = integrate.quad(lambda zz: C_CMS / cosmo.hubble(zz), 0.0, z, epsabs=0.0, epsrel=1e-12, limit=200)
    return val


def luminosity_distance(z: float, cosmo: Cosmology = PLANCK13) -> float:
    """d_L = (1 + z) int_0^z c dz' / H(z') in a flat universe (Sec. 6.1)."""
    return (1.0 + z) * comoving_distance(z, cosmo)


def angular_diameter_distance(z: float, cosmo: Cosmology = PLANCK13) -> float:
    """d_A = d_L / (1 + z)^2."""
    return luminosity_distance(z, cosmo) / (1.0 + z) ** 2


# ------------------------------------------------------------ Eq. SB units --
def sb_factor(L: float, n_packets: int, z: float, l_pix_cm: float) -> float:
    """erg s^-1 cm^-2 arcsec^-2 per unit of the peel-off sum in one pixel:
    L / [4 pi N_ph (1 + z)^4 206265^2 l_pix^2] (Sec. 6.1; l_pix is the pixel's
    physical size)."""
    return L / (4.0 * math.pi * n_packets * (1.0 + z) ** 4 * ARCSEC_PER_RAD ** 2 * l_pix_cm ** 2)


def pixel_size(fov_half_cm: float, npix: int) -> float:
    return 2.0 * fov_half_cm / npix


def surface_brightness(image, L: float, n_packets: int, z: float, fov_half_cm: float,
                       transmission=None):
    """Surface brightness (erg s^-1 cm^-2 arcsec^-2) of a camera image cube
    [npix, npix, nbins] (the colt_read_image layout, [v][u][bin]) integrated
    over frequency; transmission[nbins] (e.g. igm_transmission) weights the
    frequency bins first (Eq. SB's e^-tau_IGM)."""
    img = np.asarray(image, np.float64)
    npix = img.shape[0]
    if transmission is not None:
        img = img * np.asarray(transmission, np.float64)[None, None, :]
    return img.sum(axis=2) * sb_factor(L, n_packets, z, pixel_size(fov_half_cm, npix))


def velocity_edges(lo_kms: float, hi_kms: float, nbins: int) -> np.ndarray:
    return np.linspace(lo_kms, hi_kms, nbins + 1)


def observed_wavelength(dv_kms, z: float):
    """lambda_obs (cm) of a photon leaving the source at Doppler velocity dv
    (red positive) from redshift z."""
    return LAMBDA_LYA_CM * (1.0 + np.asarray(dv_kms, np.float64) / C_KMS) * (1.0 + z)


def flux_density(cam_spec, L: float, n_packets: int, z: float, lo_kms: float, hi_kms: float,
                 cosmo: Cosmology = PLANCK13, transmission=None):
    """f_lambda (erg s^-1 cm^-2 per cm of observed wavelength) per bin of a
    camera spectrum binned uniformly in Delta v on [lo, hi):
    sum x L / (4 pi N_ph Delta lambda_obs d_L^2), Delta lambda_obs = (1 + z)
    Delta lambda_bin (Sec. 6.1 and its footnote)."""
    s = np.asarray(cam_spec, np.float64)
    if transmission is not None:
        s = s * np.asarray(transmission, np.float64)
    e = observed_wavelength(velocity_edges(lo_kms, hi_kms, s.shape[-1]), z)
    dl = np.diff(e)
    d = luminosity_distance(z, cosmo)
    return s * L / (4.0 * math.pi * n_packets * dl * d * d)


# ----------------------------------------------------- profiles and radii --
def radial_profile(sb_map, fov_half_cm: float, nbins: int = 32):
    """Azimuthally averaged surface brightness in equal-width annuli about the
    image centre out to fov_half: (radius of each annulus centre in cm, mean SB)."""
    m = np.asarray(sb_map, np.float64)
    npix = m.shape[0]
    c = (np.arange(npix) + 0.5) * pixel_size(fov_half_cm, npix) - fov_half_cm
    r = np.hypot(c[None, :], c[:, None])
    edges = np.linspace(0.0, fov_half_cm, nbins + 1)
    idx = np.digitize(r.ravel(), edges) - 1
    ok = (idx >= 0) & (idx < nbins)
    tot = np.bincount(idx[ok], weights=m.ravel()[ok], minlength=nbins)
    cnt = np.bincount(idx[ok], minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        prof = np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)
    return 0.5 * (edges[1:] + edges[:-1]), prof


def half_light_radius(sb_map, fov_half_cm: float) -> float:
    """R_1/2 of a surface-brightness map: the radius about the image centre
    within which half of the light of the map falls (Sec. 6.1: the integrated
    light I(r) ~ int_0^r SB(r') r' dr'), from the pixel sums sorted by radius
    with linear interpolation."""
    m = np.asarray(sb_map, np.float64)
    npix = m.shape[0]
    c = (np.arange(npix) + 0.5) * pixel_size(fov_half_cm, npix) - fov_half_cm
    r = np.hypot(c[None, :], c[:, None]).ravel()
    order = np.argsort(r, kind="stable")
    cum = np.cumsum(m.ravel()[order])
    if cum[-1] <= 0:
        return float("nan")
    half = 0.5 * cum[-1]
    k = int(np.searchsorted(cum, half))
    if k == 0:
        return float(r[order[0]])
    r0, r1, c0, c1 = r[order[k - 1]], r[order[k]], cum[k - 1], cum[k]
    return float(r0 + (r1 - r0) * (half - c0) / (c1 - c0)) if c1 > c0 else float(r1)


# --------------------------------------------------- IGM damping wing --
def tau_gp_line_centre(z: float) -> float:
    """Gunn-Peterson optical depth at line centre, 7e5 ((1 + z)/10)^3/2 (Sec. 6.1)."""
    return 7.0e5 * ((1.0 + z) / 10.0) ** 1.5


def r_alpha() -> float:
    """R_alpha = Lambda lambda_alpha / (4 pi c) (~2e-8, Sec. 6.1)."""
    return A_LYA * LAMBDA_LYA_CM / (4.0 * math.pi * C_CMS)


def _wing_integral(x0: float, x1: float, ra: float) -> float:
    """int_{x0}^{x1} x^9/2 / ((1 - x)^2 + R^2 x^6) dx (x1 < 1 for red photons)."""
    if x1 <= x0:
        return 0.0
    f = lambda x: x ** 4.5 / ((1.0 - x) ** 2 + ra * ra * x ** 6)
    pts = [p for p in (1.0,) if x0 < p < x1]
    val, _ = integrate.quad(f, x0, x1, points=pts or None, epsabs=0.0, epsrel=1e-10, limit=400)
    return val


def tau_gp_red(lambda_obs_cm, z_em: float, z_i: float, z_rei: float) -> np.ndarray:
    """Eq. tauGP: red damping-wing optical depth of a neutral Einstein-de
    Sitter IGM between the reionization redshift z_rei and the edge of the
    source's HII region at z_i, for photons observed at lambda_obs:
    tau_0(z_em) R_alpha / pi [lambda_alpha (1 + z_em) / lambda_obs]^3/2
    int_{x_rei}^{x_i} x^9/2 / ((1 - x)^2 + R_alpha^2 x^6) dx, with
    x = (1 + z') lambda_alpha / lambda_obs."""
    lam = np.atleast_1d(np.asarray(lambda_obs_cm, np.float64))
    ra = r_alpha()
    pre = tau_gp_line_centre(z_em) * ra / math.pi
    out = np.empty_like(lam)
    for i, l in enumerate(lam):
        x_rei = (1.0 + z_rei) * LAMBDA_LYA_CM / l
        x_i = (1.0 + z_i) * LAMBDA_LYA_CM / l
        out[i] = pre * (LAMBDA_LYA_CM * (1.0 + z_em) / l) ** 1.5 * _wing_integral(x_rei, x_i, ra)
    return out


def igm_transmission(lo_kms: float, hi_kms: float, nbins: int, z_em: float, z_i: float, z_rei: float):
    """e^-tau_IGM at the centre of each Delta v bin (tau_IGM = tau_GP^red, Sec. 6.1)."""
    e = velocity_edges(lo_kms, hi_kms, nbins)
    return np.exp(-tau_gp_red(observed_wavelength(0.5 * (e[1:] + e[:-1]), z_em), z_em, z_i, z_rei))
