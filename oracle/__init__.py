"""FP64 CPU oracle of the Lyman-alpha packet loop (Smith et al. 2014, COLT).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the product path (the CUDA
library and its binding) never does.  The C sources share nothing with the
CUDA library.  Functions here marshal numpy arrays into liboracle.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        _LIB = C.CDLL(path)
        _setup(_LIB)
    return _LIB


class GridIn(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic_xy", C.c_int),
                ("n_HI", C.c_void_p), ("T", C.c_void_p), ("vx", C.c_void_p), ("vy", C.c_void_p),
                ("vz", C.c_void_p), ("k_dust", C.c_void_p),
                ("n_leaves", C.c_int64), ("leaf_level", C.c_void_p), ("leaf_ijk", C.c_void_p),
                ("lum", C.c_void_p)]


class Camera(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("npix", C.c_int)]


class Params(C.Structure):
    _fields_ = [("n_packets", C.c_uint64), ("seed", C.c_uint64), ("src_pos", C.c_double * 3),
                ("src_sigma", C.c_double), ("core_skip", C.c_int), ("recoil", C.c_int),
                ("phase", C.c_int), ("f_nl", C.c_double), ("tau_esc_max", C.c_double),
                ("albedo", C.c_double), ("max_scatter", C.c_uint64), ("spec_units", C.c_int),
                ("T_ref", C.c_double), ("spec_lo", C.c_double), ("spec_hi", C.c_double),
                ("spec_nbins", C.c_int), ("n_cam", C.c_int), ("cams", C.c_void_p),
                ("cam_units", C.c_int), ("cam_lo", C.c_double), ("cam_hi", C.c_double),
                ("cam_nbins", C.c_int), ("fov_half", C.c_double), ("n_threads", C.c_int),
                ("pk_status", C.c_void_p), ("pk_nscat", C.c_void_p), ("pk_freq", C.c_void_p),
                ("pid0", C.c_uint64), ("emission", C.c_int), ("source", C.c_int),
                ("n_sources", C.c_int), ("sources", C.c_void_p), ("exact", C.c_int)]


class Result(C.Structure):
    _fields_ = [("n_emitted", C.c_uint64), ("n_escaped", C.c_uint64), ("n_absorbed", C.c_uint64),
                ("n_capped", C.c_uint64), ("n_scat", C.c_uint64), ("n_scat_hi", C.c_uint64),
                ("n_cell_visits", C.c_uint64), ("n_peel_visits", C.c_uint64),
                ("spec_under", C.c_uint64), ("spec_over", C.c_uint64),
                ("spec", C.c_void_p), ("cam_spec", C.c_void_p), ("cam_spec2", C.c_void_p),
                ("cam_image", C.c_void_p), ("cam_total", C.c_void_p),
                ("n_threads_used", C.c_int), ("seconds", C.c_double), ("transport_seconds", C.c_double)]


class ScatterIO(C.Structure):
    _fields_ = [("x", C.c_double), ("k", C.c_double * 3), ("a", C.c_double), ("g", C.c_double),
                ("atau0", C.c_double), ("phase", C.c_int), ("pid", C.c_uint64), ("event", C.c_uint32),
                ("x_f", C.c_double), ("k_f", C.c_double * 3), ("u_atom", C.c_double * 3),
                ("u_par", C.c_double), ("x_crit", C.c_double), ("RQ", C.c_double), ("mu", C.c_double),
                ("n_trials", C.c_int), ("exact", C.c_int)]


def _setup(L):
    d, P, sz = C.c_double, C.c_void_p, C.c_size_t
    for name in ("o_vth_kms", "o_damping_a", "o_sigma0", "o_recoil_g", "o_x_cw_fit",
                 "o_x_cw_lambert", "o_x_crit"):
        getattr(L, name).restype = d
        getattr(L, name).argtypes = [d]
    L.o_atau_jeans.restype = d
    L.o_atau_jeans.argtypes = [d, d]
    for name in ("o_H_exact", "o_H_approx"):
        getattr(L, name).restype = d
        getattr(L, name).argtypes = [d, d]
    for name in ("o_H_exact_many", "o_H_approx_many"):
        getattr(L, name).restype = None
        getattr(L, name).argtypes = [P, P, P, sz]
    L.o_philox_many.argtypes = [P, P, P, sz]
    L.o_uniform.restype = d
    L.o_uniform.argtypes = [C.c_uint32]
    L.o_scatter_many.argtypes = [P, sz, P]
    L.o_sample_upar_many.argtypes = [d, d, C.c_uint64, C.c_uint32, P, P, P, sz]
    L.o_sample_upar_many_ex.argtypes = [d, d, C.c_uint64, C.c_uint32, P, P, P, sz, C.c_int]
    L.o_sample_mu_many.argtypes = [d, P, P, sz]
    L.o_atau_nl.restype = C.c_int
    L.o_atau_nl.argtypes = [P, d, P]
    L.o_run.restype = C.c_int
    L.o_run.argtypes = [P, P, P]
    L.o_prepare.restype = C.c_void_p
    L.o_prepare.argtypes = [P, P]
    L.o_run_prepared.restype = C.c_int
    L.o_run_prepared.argtypes = [P, P, P]
    L.o_prepared_free.restype = None
    L.o_prepared_free.argtypes = [P]
    L.o_octree_locate.restype = C.c_int64
    L.o_octree_locate.argtypes = [P, P, P]


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _key(seed: int):
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)


# ---------------------------------------------------------------- scalars --
def vth_kms(T): return lib().o_vth_kms(float(T))
def damping_a(T): return lib().o_damping_a(float(T))
def sigma0(T): return lib().o_sigma0(float(T))
def recoil_g(T): return lib().o_recoil_g(float(T))
def x_cw_fit(a): return lib().o_x_cw_fit(float(a))
def x_cw_lambert(a): return lib().o_x_cw_lambert(float(a))
def x_crit(atau0): return lib().o_x_crit(float(atau0))


def atau_jeans(T, n_HI): return lib().o_atau_jeans(float(T), float(n_HI))


def _vec2(fn, a, x):
    a, x = np.broadcast_arrays(np.asarray(a, np.float64), np.asarray(x, np.float64))
    shape = a.shape
    a = np.ascontiguousarray(a.ravel(), np.float64)
    x = np.ascontiguousarray(x.ravel(), np.float64)
    out = np.empty(a.shape, np.float64)
    fn(_ptr(a), _ptr(x), _ptr(out), a.size)
    return float(out[0]) if shape == () else out.reshape(shape)


def H_approx(a, x):
    return _vec2(lib().o_H_approx_many, a, x)


def H_exact(a, x):
    return _vec2(lib().o_H_exact_many, a, x)


def philox(ctr, key):
    """ctr: (n,4) uint32, key: (n,2) uint32 -> (n,4) uint32."""
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, np.uint32), (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    lib().o_philox_many(_ptr(ctr), _ptr(key), _ptr(out), ctr.shape[0])
    return out


def uniform(r):
    return np.array([lib().o_uniform(int(v)) for v in np.asarray(r, np.uint32).ravel()])


def sample_upar(x, a, n, seed=1, pid0=0, event=1, exact=False):
    """n draws of u_par at frequency x (packet ids pid0 + i); exact: the
    exact-physics mode (|x| >= 9 by numeric inversion of Eq. uparf)."""
    out = np.empty(n, np.float64)
    ntr = np.empty(n, np.int32)
    k = _key(seed)
    lib().o_sample_upar_many_ex(float(x), float(a), int(pid0), int(event), _ptr(k), _ptr(out), _ptr(ntr), n,
                                int(bool(exact)))
    return out, ntr


def sample_mu(RQ, u):
    u = np.ascontiguousarray(u, np.float64)
    mu = np.empty_like(u)
    lib().o_sample_mu_many(float(RQ), _ptr(u), _ptr(mu), u.size)
    return mu


SCATTER_IN = ("x", "k", "a", "g", "atau0", "phase", "pid", "event")
SCATTER_OUT = ("x_f", "k_f", "u_atom", "u_par", "x_crit", "RQ", "mu", "n_trials")


def scatter(inp: dict, seed: int) -> dict:
    """One resonant scattering per row.  inp: x (n,), k (n,3), a (n,), g (n,),
    atau0 (n,), phase (n,) int, pid (n,) uint64, event (n,) uint32."""
    n = len(inp["x"])
    arr = (ScatterIO * n)()
    npa = np.ctypeslib.as_array(arr)
    npa["x"] = inp["x"]
    npa["k"] = np.asarray(inp["k"]).reshape(n, 3)
    npa["a"] = inp["a"]
    npa["g"] = inp["g"]
    npa["atau0"] = inp["atau0"]
    npa["phase"] = inp["phase"]
    npa["pid"] = inp["pid"]
    npa["event"] = inp["event"]
    k = _key(seed)
    lib().o_scatter_many(C.cast(arr, C.c_void_p), n, _ptr(k))
    return {f: np.array(npa[f]) for f in SCATTER_OUT}


def _grid_struct(g):
    keep = []

    def P(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dt)
        keep.append(a)
        return _ptr(a)

    s = GridIn()
    s.kind = g.kind
    s.nx, s.ny, s.nz = [int(v) for v in g.shape]
    s.lo = (C.c_double * 3)(*[float(v) for v in g.lo])
    s.hi = (C.c_double * 3)(*[float(v) for v in g.hi])
    s.periodic_xy = int(bool(g.periodic_xy))
    s.n_HI = P(g.n_HI, np.float32)
    s.T = P(g.T, np.float32)
    s.vx = P(g.vx, np.float32)
    s.vy = P(g.vy, np.float32)
    s.vz = P(g.vz, np.float32)
    s.k_dust = P(g.k_dust, np.float32)
    if g.kind == 1:
        s.n_leaves = int(g.n_cells)
        s.leaf_level = P(g.leaf_level, np.uint8)
        s.leaf_ijk = P(g.leaf_ijk, np.uint32)
    s.lum = P(getattr(g, "lum", None), np.float64)
    return s, keep


def atau_nl(g, f_nl=0.5):
    s, keep = _grid_struct(g)
    out = np.zeros(g.n_cells, np.float64)
    rc = lib().o_atau_nl(C.byref(s), float(f_nl), _ptr(out))
    if rc:
        raise ValueError(f"oracle grid rejected ({rc})")
    return out


def octree_locate(g, pos, direction):
    s, keep = _grid_struct(g)
    p = np.asarray(pos, np.float64)
    d = np.asarray(direction, np.float64)
    return int(lib().o_octree_locate(C.byref(s), _ptr(p), _ptr(d)))


def _params(g, spec, n_threads, per_packet, images, pid0, exact):
    """(o_params, keep-alive list, output dict, o_result) for one run."""
    p = Params()
    p.pid0 = int(pid0) + int(getattr(spec, "pid_offset", 0) or 0)
    p.n_packets = int(spec.n_packets)
    p.seed = int(spec.seed)
    p.src_pos = (C.c_double * 3)(*[float(v) for v in spec.src_pos])
    p.src_sigma = float(spec.src_sigma)
    p.core_skip = int(spec.core_skip)
    p.recoil = int(bool(spec.recoil))
    p.phase = int(spec.phase)
    p.f_nl = float(spec.f_nl)
    p.tau_esc_max = float(spec.tau_esc_max)
    p.albedo = float(spec.albedo)
    p.max_scatter = int(spec.max_scatter)
    p.emission = int(getattr(spec, "emission", 0) or 0)
    p.source = int(getattr(spec, "source", 0) or 0)
    srcs = list(getattr(spec, "sources", None) or [])
    p.n_sources = len(srcs)
    src_arr = np.array([[*map(float, pos), float(sig), float(w)] for pos, sig, w in srcs], np.float64).reshape(-1)
    p.sources = _ptr(src_arr) if srcs else None
    p.exact = int(bool(exact))
    p.spec_units = int(spec.spec_units)
    p.T_ref = float(spec.T_ref)
    p.spec_lo, p.spec_hi, p.spec_nbins = float(spec.spec_lo), float(spec.spec_hi), int(spec.spec_nbins)
    ncam = len(spec.cameras)
    cams = (Camera * max(ncam, 1))()
    for i, cam in enumerate(spec.cameras):
        cams[i].dir = (C.c_double * 3)(*[float(v) for v in cam.direction])
        cams[i].npix = int(cam.npix) if images else 0
    p.n_cam = ncam
    p.cams = C.cast(cams, C.c_void_p)
    p.cam_units = int(spec.cam_units)
    p.cam_lo, p.cam_hi, p.cam_nbins = float(spec.cam_lo), float(spec.cam_hi), int(spec.cam_nbins)
    fov = spec.fov_half if spec.fov_half > 0 else 0.5 * float(np.max(np.asarray(g.hi) - np.asarray(g.lo)))
    p.fov_half = float(fov)
    p.n_threads = int(n_threads)
    out = {}
    keep = [cams, src_arr]
    if per_packet:
        out["pk_status"] = np.zeros(spec.n_packets, np.int32)
        out["pk_nscat"] = np.zeros(spec.n_packets, np.uint64)
        out["pk_freq"] = np.zeros(spec.n_packets, np.float64)
        p.pk_status, p.pk_nscat, p.pk_freq = (_ptr(out["pk_status"]), _ptr(out["pk_nscat"]),
                                              _ptr(out["pk_freq"]))
    r = Result()
    spec_arr = np.zeros(spec.spec_nbins, np.uint64)
    r.spec = _ptr(spec_arr)
    out["spec"] = spec_arr
    if ncam:
        cs = np.zeros((ncam, spec.cam_nbins), np.float64)
        cs2 = np.zeros((ncam, spec.cam_nbins), np.float64)
        ct = np.zeros(ncam, np.float64)
        r.cam_spec, r.cam_spec2, r.cam_total = _ptr(cs), _ptr(cs2), _ptr(ct)
        out.update(cam_spec=cs, cam_spec2=cs2, cam_total=ct)
        if images:
            npx = [int(c.npix) for c in spec.cameras]
            img = np.zeros(sum(n * n for n in npx) * spec.cam_nbins, np.float64)
            r.cam_image = _ptr(img)
            out["cam_image"] = img
    return p, keep, out, r


def _outputs(out, r):
    out.update(n_emitted=r.n_emitted, n_escaped=r.n_escaped, n_absorbed=r.n_absorbed,
               n_capped=r.n_capped, n_scat=r.n_scat, n_scat_hi=r.n_scat_hi,
               n_cell_visits=r.n_cell_visits, n_peel_visits=r.n_peel_visits,
               spec_under=r.spec_under, spec_over=r.spec_over, seconds=r.seconds,
               transport_seconds=r.transport_seconds,
               n_threads=r.n_threads_used)
    return out


def run(g, spec, n_threads: int = 0, per_packet: bool = False, images: bool = False, pid0: int = 0,
        exact: bool = False) -> dict:
    """Full packet loop on grid g with run description spec (synth.RunSpec);
    packets are ids pid0 .. pid0 + spec.n_packets - 1.  exact: the
    exact-physics mode (quadrature H, exact far-wing u_par), for measuring
    the bias of the approximations."""
    s, keep = _grid_struct(g)
    p, keep2, out, r = _params(g, spec, n_threads, per_packet, images, pid0, exact)
    rc = lib().o_run(C.byref(s), C.byref(p), C.byref(r))
    if rc:
        raise ValueError(f"oracle run rejected its inputs ({rc})")
    return _outputs(out, r)


def run_many(g, specs, images: bool = False, workers: int = 4, per_packet: bool = False) -> list:
    """Several runs on one grid derivation: the grid's cell quantities (and
    a tau_NL, luminosity weights) are derived once for specs[0], whose
    core_skip, f_nl and source every spec must share, and the runs proceed
    `workers` at a time (each on its share of the host threads), so that the
    longest histories of one run overlap the others."""
    import os
    import threading
    s, keep = _grid_struct(g)
    p0, keep0, _, _ = _params(g, specs[0], 0, False, False, 0, False)
    pg = lib().o_prepare(C.byref(s), C.byref(p0))
    if not pg:
        raise ValueError("oracle grid rejected")
    workers = max(1, min(workers, len(specs)))
    nthr = max(1, (os.cpu_count() or 1) // workers)
    results = [None] * len(specs)
    errors = []
    nxt = [0]
    mu = threading.Lock()

    def worker():
        while True:
            with mu:
                i = nxt[0]
                nxt[0] += 1
            if i >= len(specs) or errors:
                return
            p, kp, out, r = _params(g, specs[i], nthr, per_packet, images, 0, False)
            rc = lib().o_run_prepared(C.c_void_p(pg), C.byref(p), C.byref(r))
            if rc:
                errors.append(ValueError(f"oracle run rejected its inputs ({rc})"))
                return
            results[i] = _outputs(out, r)

    try:
        ths = [threading.Thread(target=worker) for _ in range(workers)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    finally:
        lib().o_prepared_free(C.c_void_p(pg))
    if errors:
        raise errors[0]
    return results
