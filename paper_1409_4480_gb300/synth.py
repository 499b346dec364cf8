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
    core_skip: bool = True
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
