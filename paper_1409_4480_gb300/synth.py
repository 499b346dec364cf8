"""Seeded synthetic inputs: grids, sources and cameras.

This module builds the per-cell fields (n_HI in cm^-3, T in K, bulk velocity
in km/s, grey dust opacity in cm^-1) and the run descriptions that both the
CUDA library and the CPU oracle consume.  It holds none of the transport
arithmetic: each side derives its own opacities, Doppler widths and damping
parameters from these raw fields.

The one physical relation used here is the workload recipe itself: a sphere or
slab "of line-centre optical depth tau0 at temperature T" is the one whose HI
density is n_HI = tau0 / (sigma_0(T) R), with sigma_0 = 5.898e-14 T4^-1/2 cm^2
(the paper's line-centre cross-section, Sec. 2) -- this is how the paper and
the workloads specify their spheres and slabs.

Geometry follows the paper's test problems:
  * static / Hubble-expanding uniform sphere (Sec. 4.2, v = v_max r / R, the
    velocity taken at the cell centre; a cell is inside when its centre is);
  * uniform slab |z| < H, periodic in x and y (Sec. 4.1, Neufeld test);
  * octree haloes and a cosmological box (synthetic stand-ins for the paper's
    simulation data, which are not available).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

PC_CM = 3.0856775814913673e18  # one parsec in cm

KIND_CARTESIAN = 0
KIND_OCTREE = 1


@dataclasses.dataclass
class Grid:
    """Raw per-cell input fields.  Arrays are float32, one entry per cell
    (Cartesian: x fastest, then y, then z; octree: one entry per leaf)."""
    kind: int
    lo: np.ndarray              # (3,) float64, cm
    hi: np.ndarray              # (3,) float64, cm
    n_HI: np.ndarray
    T: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    k_dust: np.ndarray
    shape: tuple = (0, 0, 0)    # Cartesian (nx, ny, nz)
    periodic_xy: bool = False
    leaf_level: Optional[np.ndarray] = None   # uint8  (octree)
    leaf_ijk: Optional[np.ndarray] = None     # uint32 (n_leaves, 3)
    meta: dict = dataclasses.field(default_factory=dict)
    lum: Optional[np.ndarray] = None          # float64 per-cell luminosity (diffuse emission)

    @property
    def n_cells(self) -> int:
        return int(self.n_HI.shape[0])


@dataclasses.dataclass
class Camera:
    direction: tuple            # unit coordinate axis, e.g. (1, 0, 0)
    npix: int = 0               # pixels per side (0 = spectrum only)


def axis_cameras(npix: int, axes: Sequence[str] = ("+x", "-x", "+y", "-y", "+z", "-z")) -> List[Camera]:
    table = {"+x": (1.0, 0.0, 0.0), "-x": (-1.0, 0.0, 0.0), "+y": (0.0, 1.0, 0.0),
             "-y": (0.0, -1.0, 0.0), "+z": (0.0, 0.0, 1.0), "-z": (0.0, 0.0, -1.0)}
    return [Camera(table[a], npix) for a in axes]


@dataclasses.dataclass
class RunSpec:
    """Parameters of one radiative-transfer solve (mirrors colt_run_params)."""
    n_packets: int
    seed: int
    src_pos: tuple = (0.0, 0.0, 0.0)
    src_sigma: float = 0.0
    core_skip: int = 1              # 0 off, 1 a tau_cell + a tau_NL, 2 Jeans estimate
    recoil: bool = True
    phase: int = 0                  # 0 dipole/anisotropic, 1 isotropic
    f_nl: float = 0.5
    tau_esc_max: float = 50.0
    albedo: float = 0.32
    max_scatter: int = 10**9
    spec_units: int = 0             # 0: x at T_ref, 1: Delta v (km/s)
    T_ref: float = 1.0e4
    spec_lo: float = -40.0
    spec_hi: float = 40.0
    spec_nbins: int = 100
    cameras: List[Camera] = dataclasses.field(default_factory=list)
    cam_units: int = 1
    cam_lo: float = -1000.0
    cam_hi: float = 1000.0
    cam_nbins: int = 200
    fov_half: float = 0.0           # 0 -> half of the box width
    precision: int = 1              # 0 plain FP64, 1 mixed (FP32 transport)
    pid_offset: int = 0             # packets are ids pid_offset .. pid_offset + n_packets - 1
    emission: int = 0               # 0 line centre, 1 natural (Lorentzian) + thermal atom velocity
    source: int = 0                 # 0 point (src_pos, src_sigma), 1 cells by luminosity (Grid.lum)
    sources: list = dataclasses.field(default_factory=list)   # [(pos, sigma, weight)]: several point sources


def sigma0_recipe(T: float) -> float:
    """Line-centre cross-section used to turn a workload's tau0 into n_HI."""
    return 5.898e-14 / math.sqrt(T / 1.0e4)


def _cell_centres(n: int, lo: float, hi: float) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def sphere(n: int, T: float, tau0: float, R: float = PC_CM, v_max_kms: float = 0.0,
           tau_dust: float = 0.0) -> Grid:
    """Uniform HI sphere of radius R filling the box [-R, R]^3 on an n^3 grid.

    Inside (cell centre r < R): n_HI = tau0 / (sigma_0 R), temperature T,
    Hubble-like velocity v = v_max r / R (Sec. 4.2), dust opacity tau_dust / R.
    Outside: empty, same temperature, at rest, no dust."""
    c = _cell_centres(n, -R, R)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    inside = r < R
    nH = np.where(inside, tau0 / (sigma0_recipe(T) * R), 0.0)
    vs = np.where(inside, v_max_kms / R, 0.0)
    kd = np.where(inside, tau_dust / R, 0.0)
    g = Grid(kind=KIND_CARTESIAN, lo=np.array([-R, -R, -R]), hi=np.array([R, R, R]),
             n_HI=nH.ravel().astype(np.float32), T=np.full(n ** 3, T, np.float32),
             vx=(vs * x).ravel().astype(np.float32), vy=(vs * y).ravel().astype(np.float32),
             vz=(vs * z).ravel().astype(np.float32), k_dust=kd.ravel().astype(np.float32),
             shape=(n, n, n))
    g.meta = dict(model="sphere", n=n, T=T, tau0=tau0, R=R, v_max_kms=v_max_kms, tau_dust=tau_dust)
    return g


def slab(n: int, T: float, tau0: float, H: float = PC_CM, v_max_kms: float = 0.0,
         tau_dust: float = 0.0, nxy: Optional[int] = None) -> Grid:
    """Uniform slab |z| < H, periodic in x and y (the infinite slab of the
    Neufeld test, Sec. 4.1).  The box is [-H, H] in every axis; n cells along
    z and nxy (default n) along x and y.  Velocity v_z = v_max z / H."""
    nxy = n if nxy is None else nxy
    cz = _cell_centres(n, -H, H)
    nH = np.full((n, nxy, nxy), tau0 / (sigma0_recipe(T) * H))
    vz = np.broadcast_to((v_max_kms / H) * cz[:, None, None], (n, nxy, nxy))
    g = Grid(kind=KIND_CARTESIAN, lo=np.array([-H, -H, -H]), hi=np.array([H, H, H]),
             n_HI=nH.ravel().astype(np.float32), T=np.full(n * nxy * nxy, T, np.float32),
             vx=np.zeros(n * nxy * nxy, np.float32), vy=np.zeros(n * nxy * nxy, np.float32),
             vz=np.ascontiguousarray(vz).ravel().astype(np.float32),
             k_dust=np.full(n * nxy * nxy, tau_dust / H, np.float32),
             shape=(nxy, nxy, n), periodic_xy=True)
    g.meta = dict(model="slab", n=n, T=T, tau0=tau0, H=H, v_max_kms=v_max_kms, tau_dust=tau_dust)
    return g


def uniform_box(shape, lo, hi, n_HI, T, v=(0.0, 0.0, 0.0), k_dust=0.0, periodic_xy=False) -> Grid:
    """Homogeneous Cartesian box (used by small analytic tests)."""
    nx, ny, nz = shape
    m = nx * ny * nz
    return Grid(kind=KIND_CARTESIAN, lo=np.asarray(lo, np.float64), hi=np.asarray(hi, np.float64),
                n_HI=np.full(m, n_HI, np.float32), T=np.full(m, T, np.float32),
                vx=np.full(m, v[0], np.float32), vy=np.full(m, v[1], np.float32),
                vz=np.full(m, v[2], np.float32), k_dust=np.full(m, k_dust, np.float32),
                shape=(nx, ny, nz), periodic_xy=periodic_xy)


def random_fields(shape, seed: int, lo=-PC_CM, hi=PC_CM, n_range=(1e-2, 10.0), T_range=(10.0, 1e4),
                  v_kms=30.0, k_dust_max=0.0) -> Grid:
    """Cartesian grid with independent log-uniform density and temperature and
    Gaussian velocities per cell (structure-free stress input for parity)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    m = nx * ny * nz
    ln = rng.uniform(math.log(n_range[0]), math.log(n_range[1]), m)
    lt = rng.uniform(math.log(T_range[0]), math.log(T_range[1]), m)
    return Grid(kind=KIND_CARTESIAN, lo=np.array([lo] * 3, np.float64), hi=np.array([hi] * 3, np.float64),
                n_HI=np.exp(ln).astype(np.float32), T=np.exp(lt).astype(np.float32),
                vx=rng.normal(0, v_kms, m).astype(np.float32), vy=rng.normal(0, v_kms, m).astype(np.float32),
                vz=rng.normal(0, v_kms, m).astype(np.float32),
                k_dust=rng.uniform(0, k_dust_max, m).astype(np.float32), shape=(nx, ny, nz))


# ------------------------------------------------------------------ octrees --
def octree_refine(lo, hi, refine, min_level: int, max_level: int):
    """Leaves of an octree over the box [lo, hi).

    Starts from every node of the uniform level min_level and splits each node
    for which refine(centre (m, 3), size (m, 3), level) is true, down to
    max_level.  Returns (leaf_level uint8 (n,), leaf_ijk uint32 (n, 3)); leaf i
    spans lo + ijk (hi - lo) 2^-level .. lo + (ijk + 1) (hi - lo) 2^-level, and
    the leaves tile the box.  Order: level by level, x fastest within a level."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    n0 = 1 << min_level
    kk, jj, ii = np.meshgrid(np.arange(n0), np.arange(n0), np.arange(n0), indexing="ij")
    ijk = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.int64)
    offs = np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.int64)
    levels, leaves = [], []
    for L in range(min_level, max_level + 1):
        size = (hi - lo) / float(1 << L)
        if L < max_level and len(ijk):
            split = np.asarray(refine(lo + (ijk + 0.5) * size, np.broadcast_to(size, ijk.shape), L), bool)
        else:
            split = np.zeros(len(ijk), bool)
        keep = ijk[~split]
        levels.append(np.full(len(keep), L, np.uint8))
        leaves.append(keep)
        ijk = (2 * ijk[split][:, None, :] + offs[None, :, :]).reshape(-1, 3)
        if not len(ijk):
            break
    return np.concatenate(levels), np.concatenate(leaves).astype(np.uint32)


def leaf_geometry(lo, hi, leaf_level, leaf_ijk):
    """Centres and sizes (n, 3) of octree leaves."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    size = (hi - lo)[None, :] / np.exp2(leaf_level.astype(np.float64))[:, None]
    return lo[None, :] + (leaf_ijk.astype(np.float64) + 0.5) * size, size


def octree_grid(lo, hi, leaf_level, leaf_ijk, fields) -> Grid:
    """Octree Grid from leaves and a dict of per-leaf fields (n_HI, T, vx,
    vy, vz, k_dust; missing velocities and dust are zero)."""
    n = len(leaf_level)
    z = np.zeros(n, np.float32)
    f32 = lambda k: np.asarray(fields[k], np.float32) if k in fields else z
    return Grid(kind=KIND_OCTREE, lo=np.asarray(lo, np.float64), hi=np.asarray(hi, np.float64),
                n_HI=f32("n_HI"), T=f32("T"), vx=f32("vx"), vy=f32("vy"), vz=f32("vz"), k_dust=f32("k_dust"),
                leaf_level=np.ascontiguousarray(leaf_level, np.uint8),
                leaf_ijk=np.ascontiguousarray(leaf_ijk, np.uint32).reshape(-1, 3))


def octree_from_cartesian(g: Grid, seed: Optional[int] = None) -> Grid:
    """The same cells as a Cartesian 2^L cube, stored as octree leaves of
    level L (optionally in a seeded random leaf order)."""
    nx, ny, nz = g.shape
    L = int(round(math.log2(nx)))
    if not (nx == ny == nz == 1 << L) or g.periodic_xy:
        raise ValueError("needs an open 2^L cube")
    c = np.arange(g.n_cells)
    ijk = np.stack([c % nx, (c // nx) % ny, c // (nx * ny)], axis=1).astype(np.uint32)
    order = np.random.default_rng(seed).permutation(g.n_cells) if seed is not None else c
    fields = {k: getattr(g, k)[order] for k in ("n_HI", "T", "vx", "vy", "vz", "k_dust")}
    out = octree_grid(g.lo, g.hi, np.full(g.n_cells, L, np.uint8)[order], ijk[order], fields)
    out.meta = dict(g.meta, octree_of="cartesian", level=L, order_seed=seed)
    return out


def octree_sphere(T: float, tau0: float, R: float = PC_CM, v_max_kms: float = 0.0, tau_dust: float = 0.0,
                  min_level: int = 3, max_level: int = 6) -> Grid:
    """The uniform sphere of sphere() on an octree refined to max_level where a
    leaf straddles the sphere surface (|r_centre - R| < leaf diagonal), and
    kept at min_level elsewhere; fields at leaf centres as in sphere()."""
    lo, hi = np.array([-R] * 3), np.array([R] * 3)

    def refine(c, s, L):
        return np.abs(np.linalg.norm(c, axis=1) - R) < np.linalg.norm(s, axis=1)

    lv, ijk = octree_refine(lo, hi, refine, min_level, max_level)
    c, _ = leaf_geometry(lo, hi, lv, ijk)
    r = np.linalg.norm(c, axis=1)
    inside = r < R
    vs = np.where(inside, v_max_kms / R, 0.0)
    g = octree_grid(lo, hi, lv, ijk, dict(
        n_HI=np.where(inside, tau0 / (sigma0_recipe(T) * R), 0.0), T=np.full(len(lv), T),
        vx=vs * c[:, 0], vy=vs * c[:, 1], vz=vs * c[:, 2], k_dust=np.where(inside, tau_dust / R, 0.0)))
    g.meta = dict(model="octree_sphere", T=T, tau0=tau0, R=R, v_max_kms=v_max_kms, tau_dust=tau_dust,
                  min_level=min_level, max_level=max_level)
    return g


MSUN_G = 1.98847e33
M_P_G = 1.67262192e-24
E_LYA_ERG = 1.634e-11        # 10.2 eV


def lya_luminosity(n_h, x_hi, T, volume):
    """Per-cell Ly-alpha luminosity (erg/s) of gas with hydrogen density n_h
    (cm^-3), neutral fraction x_hi and temperature T (K), in cells of the given
    volume (cm^3): the two mechanisms of Sec. 3.1.1 for a hydrogen-only gas
    with n_e = n_p = (1 - x_hi) n_h.
      recombination: 0.68 E_Lya alpha_B n_e n_p, with the case-B coefficient
        alpha_B ~ 2.5e-13 T4^-3/4 cm^3/s of Sec. 5.1 and the 0.68 Ly-alpha
        photons per recombination of Sec. 5.3;
      collisional excitation: 7.5e-19 erg cm^3/s (1 + T5^1/2)^-1 e^(-118348/T)
        n_e n_HI (Sec. 5.3, after Cen 1992; the excited atoms are the neutral
        ones, n_HI = x_hi n_h)."""
    n_h, x_hi, T = (np.asarray(v, np.float64) for v in (n_h, x_hi, T))
    n_e = (1.0 - x_hi) * n_h
    alpha_b = 2.5e-13 * (T / 1e4) ** -0.75
    rec = 0.68 * E_LYA_ERG * alpha_b * n_e * n_e
    col = 7.5e-19 / (1.0 + np.sqrt(T / 1e5)) * np.exp(-118348.0 / T) * n_e * x_hi * n_h
    return (rec + col) * np.asarray(volume, np.float64)


def halo(seed: int = 3, r_vir: float = 600.0 * PC_CM, m_vir_msun: float = 1e8, conc: float = 5.0,
         f_baryon: float = 0.157, x_h: float = 0.76, cone_half_angle_deg: float = 30.0,
         clump_sigma: float = 1.0, turb_kms: float = 10.0, min_level: int = 6, max_level: int = 12,
         cone_level: int = 9, leaf_mass_frac: float = 3e-6, emission: bool = False) -> Grid:
    """Synthetic first-galaxy halo on an octree (stand-in for the paper's AMR
    halo, whose simulation data are not available).

    Box +-2 r_vir.  Gas: f_baryon times an NFW profile of mass m_vir inside
    r_vir and concentration conc (rho(r) ~ 1 / ((r/r_s)(1 + r/r_s)^2),
    r_s = r_vir / conc), hydrogen mass fraction x_h, taken at the leaf centre
    (at least half a leaf size from the centre).  Inside a bicone of half angle
    cone_half_angle_deg about z: T = 1e4 K and x_HI = 1e-4; outside: T = 100 K,
    neutral.  Clumping: each leaf's density times exp(sigma G - sigma^2/2),
    G ~ N(0, 1) per leaf (mean preserving).  Turbulence: independent Gaussian
    velocity of turb_kms per component per leaf.  No dust.
    Refinement: a node splits while its gas mass exceeds leaf_mass_frac of the
    gas mass inside r_vir (down to max_level), or while it straddles the cone
    surface inside r_vir (down to cone_level), starting from min_level.
    emission: also set the per-leaf Ly-alpha luminosity of the gas
    (lya_luminosity: recombination and collisional excitation), for diffuse
    emission."""
    rng = np.random.default_rng(seed)
    R = 2.0 * r_vir
    lo, hi = np.array([-R] * 3), np.array([R] * 3)
    r_s = r_vir / conc
    m_c = math.log(1.0 + conc) - conc / (1.0 + conc)
    rho_s = m_vir_msun * MSUN_G / (4.0 * math.pi * r_s ** 3 * m_c)
    m_gas = f_baryon * m_vir_msun * MSUN_G
    cos_cone = math.cos(math.radians(cone_half_angle_deg))

    def rho_gas(c, s):
        r = np.maximum(np.linalg.norm(c, axis=1), 0.5 * s[:, 0])
        q = r / r_s
        return f_baryon * rho_s / (q * (1.0 + q) ** 2)

    def refine(c, s, L):
        mass = rho_gas(c, s) * s[:, 0] * s[:, 1] * s[:, 2]
        r = np.linalg.norm(c, axis=1)
        half_diag = 0.5 * np.linalg.norm(s, axis=1)
        # straddles the cone surface |z| = r cos(theta_c): the surface passes within the leaf
        dist = np.abs(np.abs(c[:, 2]) * math.sin(math.acos(cos_cone))
                      - np.hypot(c[:, 0], c[:, 1]) * cos_cone)
        return (mass > leaf_mass_frac * m_gas) | ((dist < half_diag) & (r < r_vir) & (L < cone_level))

    lv, ijk = octree_refine(lo, hi, refine, min_level, max_level)
    c, s = leaf_geometry(lo, hi, lv, ijk)
    n = len(lv)
    r = np.linalg.norm(c, axis=1)
    in_cone = np.abs(c[:, 2]) > cos_cone * r
    clump = np.exp(clump_sigma * rng.standard_normal(n) - 0.5 * clump_sigma ** 2)
    n_h = x_h * rho_gas(c, s) * clump / M_P_G
    x_hi = np.where(in_cone, 1e-4, 1.0)
    g = octree_grid(lo, hi, lv, ijk, dict(
        n_HI=n_h * x_hi, T=np.where(in_cone, 1e4, 100.0),
        vx=rng.normal(0.0, turb_kms, n), vy=rng.normal(0.0, turb_kms, n), vz=rng.normal(0.0, turb_kms, n)))
    g.meta = dict(model="halo", seed=seed, r_vir=r_vir, m_vir_msun=m_vir_msun, conc=conc, f_baryon=f_baryon,
                  cone_half_angle_deg=cone_half_angle_deg, clump_sigma=clump_sigma, turb_kms=turb_kms,
                  min_level=min_level, max_level=max_level, cone_level=cone_level, leaf_mass_frac=leaf_mass_frac,
                  n_leaves=n)
    if emission:
        g.lum = lya_luminosity(n_h, x_hi, np.where(in_cone, 1e4, 100.0), s[:, 0] * s[:, 1] * s[:, 2])
    return g


# ------------------------------------------------ idealized first galaxies --
# Sec. 5.1: cored isothermal hydrogen profile inside a neutral IGM, an early
# (Stromgren sphere) or late (plus a bicone) ionized region, static or
# radiation-driven wind, T = 1e4 K, on an octree refined by the Jeans, Sobolev
# and geometric criteria.  Planck 2013 parameters as Sec. 5.1 prints them.
H0_KMS_MPC, OMEGA_B, X_HYDROGEN = 67.8, 0.0485, 0.75
G_CGS = 6.67430e-8
M_H_G = 1.6735575e-24          # hydrogen atom
MPC_CM = 1e6 * PC_CM
K_B_CGS = 1.380649e-16


def n_h_igm(z: float) -> float:
    """Background hydrogen density rho_cr,0 X Omega_b (1 + z)^3 / m_H (cm^-3)."""
    h0 = H0_KMS_MPC * 1e5 / MPC_CM
    rho_cr0 = 3.0 * h0 * h0 / (8.0 * math.pi * G_CGS)
    return rho_cr0 * X_HYDROGEN * OMEGA_B * (1.0 + z) ** 3 / M_H_G


def galaxy_chi(m_h_tot_msun: float, r_core: float, z: float) -> float:
    """chi = n_IGM^(-1/3) / r_core (M_H,tot / (4 pi m_H))^(1/3) (Eq. chi)."""
    return n_h_igm(z) ** (-1.0 / 3.0) / r_core * (m_h_tot_msun * MSUN_G / (4.0 * math.pi * M_H_G)) ** (1.0 / 3.0)


def galaxy_core_density(m_h_tot_msun: float, r_core: float, z: float) -> float:
    """n_H,0 normalising the profile to M_H,tot exactly: with y = (n_0/n_IGM)^1/2,
    Eq. MHtot reads y^3 - (2/3) y^2 = chi^3 (solved by Newton's method from y = chi)."""
    c3 = galaxy_chi(m_h_tot_msun, r_core, z) ** 3
    y = max(1.0, c3 ** (1.0 / 3.0))
    for _ in range(100):
        f = y ** 3 - (2.0 / 3.0) * y * y - c3
        y_new = y - f / (3.0 * y * y - (4.0 / 3.0) * y)
        if abs(y_new - y) <= 1e-15 * y:
            y = y_new
            break
        y = y_new
    return n_h_igm(z) * y * y


def jeans_length(T, n_h):
    """lambda_J = sqrt(15 k T / (4 pi G mu rho)), mu = 1.23 m_H, rho = m_H n_H / X (Sec. 3.2.4)."""
    rho = M_H_G * np.asarray(n_h, np.float64) / X_HYDROGEN
    return np.sqrt(15.0 * K_B_CGS * np.asarray(T, np.float64) / (4.0 * math.pi * G_CGS * 1.23 * M_H_G * rho))


def galaxy(model: str, m_h_tot_msun: float, z: float = 10.0, r_core: float = 10.0 * PC_CM,
           T: float = 1e4, v_inf_kms: float = 10.0, r_star: float = PC_CM, cone_half_angle_deg: float = 30.0,
           n_jeans: int = 64, n_sobolev: int = 32, n_geo: int = 64, n_cone: int = 512,
           min_level: int = 4, max_level: int = 20) -> Grid:
    """Idealized first galaxy of Sec. 5.1 on an octree; model is one of "SE",
    "SL", "WE", "WL" (Static / Wind, Early / Late).

    n_H: n_H,0 for r <= r_core, n_H,0 (r / r_core)^-2 out to r_edge =
    r_core (n_H,0 / n_IGM)^1/2, n_IGM beyond (Eq. nHprofile), with n_H,0 from
    M_H,tot (Eq. MHtot).  Early: no neutral hydrogen inside the Stromgren
    sphere R_S = r_core; Late: also none inside the bicone of half-angle 30 deg
    about z out to r_edge.  Wind: v = v_inf (1 - R_*/r)^1/2 radially (Eq. wind)
    beyond R_*.  T uniform.  Box (-2 r_edge, 2 r_edge)^3.  Refinement
    (Sec. 5.1.4): split a node while its size exceeds lambda_J / n_jeans at its
    centre density, or (wind) the Sobolev length v_th / |dv/dr| / n_sobolev, or
    while it holds a point of the sphere r = r_edge or r = r_core and is larger
    than that radius / n_geo, or (late) while it straddles the cone surface
    inside r_edge and is larger than r_edge / n_cone.  Fields at leaf centres.
    The models are built at z = 10 (Sec. 5.1: "at redshift z ~ 10"; this
    reproduces the printed edge radii 1.09, 2.35, 5.05 and 10.88 kpc of the
    5- to 8-models) and observed at z = 9 (the flux tables).  The Sobolev
    criterion applies only outside the Stromgren sphere, where gas can be
    neutral (at R_* the wind's gradient diverges)."""
    if model not in ("SE", "SL", "WE", "WL"):
        raise ValueError("model must be SE, SL, WE or WL")
    wind, late = model[0] == "W", model[1] == "L"
    n_igm = n_h_igm(z)
    n0 = galaxy_core_density(m_h_tot_msun, r_core, z)
    r_edge = r_core * math.sqrt(n0 / n_igm)
    R = 2.0 * r_edge
    lo, hi = np.array([-R] * 3), np.array([R] * 3)
    cos_c, sin_c = math.cos(math.radians(cone_half_angle_deg)), math.sin(math.radians(cone_half_angle_deg))
    vth = 12.85e5 * math.sqrt(T / 1e4)          # cm/s (Sec. 2)

    def n_of(r):
        return np.where(r <= r_core, n0, np.where(r < r_edge, n0 * (r_core / np.maximum(r, r_core)) ** 2, n_igm))

    def refine(c, s, L):
        r = np.linalg.norm(c, axis=1)
        h = s[:, 0]
        half_diag = 0.5 * np.linalg.norm(s, axis=1)
        out = h * n_jeans > jeans_length(T, n_of(r))
        if wind:
            # only where the gas can be neutral (outside the Stromgren sphere)
            rr = np.maximum(r, r_star * (1.0 + 1e-9))
            dvdr = v_inf_kms * 1e5 * 0.5 / np.sqrt(1.0 - r_star / rr) * r_star / rr ** 2
            out |= (r + half_diag > r_core) & (h * n_sobolev * dvdr > vth)
        for rx in (r_edge, r_core):
            out |= (np.abs(r - rx) < half_diag) & (h * n_geo > rx)
        if late:
            dist = np.abs(np.abs(c[:, 2]) * sin_c - np.hypot(c[:, 0], c[:, 1]) * cos_c)
            out |= (dist < half_diag) & (r < r_edge + half_diag) & (h * n_cone > r_edge)
        return out

    lv, ijk = octree_refine(lo, hi, refine, min_level, max_level)
    c, s = leaf_geometry(lo, hi, lv, ijk)
    r = np.linalg.norm(c, axis=1)
    n_h = n_of(r)
    ionized = r < r_core                                  # Stromgren sphere, R_S = r_core
    if late:
        ionized |= (np.abs(c[:, 2]) > cos_c * r) & (r < r_edge)
    n_hi = np.where(ionized, 0.0, n_h)
    fields = dict(n_HI=n_hi, T=np.full(len(lv), T))
    if wind:
        rs = np.maximum(r, 1e-300)
        v = np.where(r > r_star, v_inf_kms * np.sqrt(np.clip(1.0 - r_star / rs, 0.0, None)), 0.0)
        for a, k in enumerate(("vx", "vy", "vz")):
            fields[k] = v * c[:, a] / rs
    g = octree_grid(lo, hi, lv, ijk, fields)
    g.meta = dict(model=f"{model}{int(round(math.log10(m_h_tot_msun)))}", m_h_tot_msun=m_h_tot_msun, z=z,
                  r_core=r_core, r_edge=r_edge, n_h0=n0, n_h_igm=n_igm, T=T, v_inf_kms=v_inf_kms, r_star=r_star,
                  cone_half_angle_deg=cone_half_angle_deg, n_jeans=n_jeans, n_sobolev=n_sobolev, n_geo=n_geo,
                  n_cone=n_cone, n_leaves=len(lv), levels=(int(lv.min()), int(lv.max())))
    return g


def _trilinear(field: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Periodic trilinear interpolation of field[z, y, x] at fractional grid
    coordinates u (m, 3) = (x, y, z) in units of the grid spacing (cell centres
    at integer + 0.5)."""
    n = field.shape[0]
    g = u - 0.5
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    out = np.zeros(len(u))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
                out += w * field[(i0[:, 2] + dz) % n, (i0[:, 1] + dy) % n, (i0[:, 0] + dx) % n]
    return out


def cosmo_box(seed: int = 5, n_fft: int = 256, box_cmpc: float = 1.0, z: float = 10.0, sigma_g: float = 2.0,
              slope: float = -2.5, min_level: int = 7, max_level: int = 14, leaf_mass_frac: float = 4e-7,
              n_sources: int = 5):
    """Synthetic cosmological volume on an octree (stand-in for the paper's
    1 Mpc^3 post-processing box, whose simulation is not available).

    A Gaussian field G with power spectrum P(k) ~ k^slope is drawn on an
    n_fft^3 periodic FFT grid (seeded), scaled to standard deviation sigma_g,
    and turned into the lognormal overdensity 1 + delta = exp(G - sigma_g^2/2).
    The box is box_cmpc comoving Mpc at redshift z (physical side
    box / (1 + z)).  Hydrogen density n_H = 1.9e-7 (1 + z)^3 (1 + delta) cm^-3.
    Stated relations: T = 200 K (1 + delta)^0.6 clipped to [10, 1e5] K;
    x_HI = (1 + delta) / (1 + delta + 0.1).  Peculiar velocities from the linear
    continuity relation on the Gaussian field, v_k = i a H f G_k k / k^2 (k
    comoving; = i H f G_k q / q^2 with q = k / a the physical wavenumber),
    f = 1, H(z) = 70 km/s/Mpc sqrt(0.3 (1+z)^3 + 0.7).  Fields are
    interpolated trilinearly to leaf centres.  No dust.
    Refinement: from the uniform level min_level, a leaf splits while its
    hydrogen mass exceeds leaf_mass_frac of the box's, down to max_level.
    Returns (grid, sources): the n_sources highest-overdensity points of the
    FFT grid (cell centres, cm, box-centred), highest first."""
    rng = np.random.default_rng(seed)
    L = box_cmpc * 3.0856775814913673e24 / (1.0 + z)        # physical side, cm
    half = 0.5 * L
    k1 = np.fft.fftfreq(n_fft) * n_fft
    kz, ky, kx = np.meshgrid(k1, k1, k1[: n_fft // 2 + 1], indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = np.power(k2, slope / 4.0)
    amp[0, 0, 0] = 0.0
    noise = rng.standard_normal((n_fft, n_fft, n_fft))
    gk = np.fft.rfftn(noise) * amp
    G = np.fft.irfftn(gk, s=(n_fft,) * 3)
    scale = sigma_g / G.std()
    G *= scale
    gk *= scale
    one_delta = np.exp(G - 0.5 * sigma_g ** 2)
    hz = 70.0 * math.sqrt(0.3 * (1.0 + z) ** 3 + 0.7) / 3.0856775814913673e19   # 1/s
    qphys = 2.0 * math.pi / L                                                    # per grid wavenumber, 1/cm
    vel = []
    for kc in (kx, ky, kz):
        vk = 1j * hz * gk * (kc * qphys) / (k2 * qphys * qphys)
        vk[0, 0, 0] = 0.0
        vel.append(np.fft.irfftn(vk, s=(n_fft,) * 3) / 1e5)                     # km/s
    lo, hi = np.array([-half] * 3), np.array([half] * 3)
    nh_mean = 1.9e-7 * (1.0 + z) ** 3
    m_box = nh_mean * L ** 3

    def refine(c, s, lev):
        u = (c - lo) / (hi - lo) * n_fft
        return nh_mean * _trilinear(one_delta, u) * s[:, 0] * s[:, 1] * s[:, 2] > leaf_mass_frac * m_box

    lv, ijk = octree_refine(lo, hi, refine, min_level, max_level)
    c, _ = leaf_geometry(lo, hi, lv, ijk)
    u = (c - lo) / (hi - lo) * n_fft
    od = _trilinear(one_delta, u)
    T = np.clip(200.0 * od ** 0.6, 10.0, 1e5)
    x_hi = od / (od + 0.1)
    g = octree_grid(lo, hi, lv, ijk, dict(n_HI=nh_mean * od * x_hi, T=T, vx=_trilinear(vel[2], u),
                                          vy=_trilinear(vel[1], u), vz=_trilinear(vel[0], u)))
    top = np.argsort(one_delta.ravel())[::-1][:n_sources]
    iz, iy, ix = np.unravel_index(top, one_delta.shape)
    src = np.stack([ix, iy, iz], axis=1) + 0.5
    sources = [tuple(lo + s / n_fft * (hi - lo)) for s in src]
    g.meta = dict(model="cosmo_box", seed=seed, n_fft=n_fft, box_cmpc=box_cmpc, z=z, sigma_g=sigma_g, slope=slope,
                  min_level=min_level, max_level=max_level, leaf_mass_frac=leaf_mass_frac, n_leaves=len(lv))
    return g, sources
