"""Python binding of libcolt (include/colt.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
transport arithmetic of its own.  The library must be present (built by
`paper_1409_4480_gb300.build`); there is no fallback: a missing or unloadable
libcolt.so raises at import of the first call.

Inputs may be numpy arrays (host memory) or torch CUDA tensors (device
memory: their data_ptr() is passed with COLT_MEM_DEVICE).  PyTorch is used
only for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

COLT_OK, COLT_EINVAL, COLT_ENOMEM, COLT_EAGAIN, COLT_ETIMEOUT, COLT_ECUDA, COLT_ENOTFOUND, COLT_EDEVICE = \
    0, -1, -2, -3, -4, -5, -6, -7
COLT_CARTESIAN, COLT_OCTREE = 0, 1
COLT_MEM_HOST, COLT_MEM_DEVICE = 0, 1
COLT_PLAIN, COLT_MIXED = 0, 1
COLT_SKIP_OFF, COLT_SKIP_CELL_NL, COLT_SKIP_JEANS = 0, 1, 2
COLT_SOURCE_POINT, COLT_SOURCE_CELLS = 0, 1

EXPORTS = ["colt_init", "colt_finalize", "colt_last_error", "colt_device_info", "colt_create_grid",
           "colt_destroy_grid", "colt_read_cells", "colt_run", "colt_run_batch", "colt_solve", "colt_submit", "colt_submit_many", "colt_poll",
           "colt_wait", "colt_read_spectrum", "colt_read_image", "colt_read_result", "colt_release", "colt_voigt", "colt_scatter",
           "colt_run_noalloc", "colt_autotune", "colt_set_cell_luminosity", "colt_cancel",
           "colt_set_launch_config"]

_LIB = None


class ColtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libcolt error {code}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic_xy", C.c_int),
                ("n_cells", C.c_int64), ("leaf_level", C.c_void_p), ("leaf_ijk", C.c_void_p),
                ("n_HI", C.c_void_p), ("T", C.c_void_p), ("vx", C.c_void_p), ("vy", C.c_void_p),
                ("vz", C.c_void_p), ("k_dust", C.c_void_p), ("fields_mem", C.c_int), ("f_nl", C.c_double)]


class Camera(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("npix", C.c_int)]


class RunParams(C.Structure):
    _fields_ = [("n_packets", C.c_uint64), ("seed", C.c_uint64), ("src_pos", C.c_double * 3),
                ("src_sigma", C.c_double), ("core_skip", C.c_int), ("recoil", C.c_int), ("phase", C.c_int),
                ("tau_esc_max", C.c_double), ("albedo", C.c_double), ("max_scatter", C.c_uint64),
                ("spec_units", C.c_int), ("T_ref", C.c_double), ("spec_lo", C.c_double),
                ("spec_hi", C.c_double), ("spec_nbins", C.c_int), ("n_cam", C.c_int), ("cams", C.c_void_p),
                ("cam_units", C.c_int), ("cam_lo", C.c_double), ("cam_hi", C.c_double), ("cam_nbins", C.c_int),
                ("fov_half", C.c_double), ("precision", C.c_int), ("block_size", C.c_int),
                ("blocks_per_sm", C.c_int), ("pid_offset", C.c_uint64), ("emission", C.c_int),
                ("source", C.c_int), ("n_sources", C.c_int), ("sources", C.c_void_p)]


class Source(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("sigma", C.c_double), ("weight", C.c_double)]


class Result(C.Structure):
    _fields_ = [("n_emitted", C.c_uint64), ("n_escaped", C.c_uint64), ("n_absorbed", C.c_uint64),
                ("n_capped", C.c_uint64), ("n_scat", C.c_uint64), ("n_scat_hi", C.c_uint64),
                ("n_cell_visits", C.c_uint64), ("n_peel_visits", C.c_uint64), ("n_peel_rays", C.c_uint64),
                ("spec_under", C.c_uint64), ("spec_over", C.c_uint64), ("kernel_ms", C.c_double),
                ("spec", C.c_void_p), ("cam_spec", C.c_void_p), ("cam_spec2", C.c_void_p),
                ("cam_image", C.c_void_p), ("pk_status", C.c_void_p), ("pk_nscat", C.c_void_p),
                ("pk_freq", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("done", C.c_int), ("admitted", C.c_int), ("packets_done", C.c_uint64),
                ("packets_total", C.c_uint64), ("submit_to_done_ms", C.c_double),
                ("ctx_launches", C.c_uint64), ("cancelled", C.c_int), ("ctx_timed_launches", C.c_uint64),
                ("ctx_kernel_ms", C.c_double), ("longest_history", C.c_uint64),
                ("ctx_cell_visits", C.c_uint64), ("ctx_peel_visits", C.c_uint64)]


class LaunchConfig(C.Structure):
    _fields_ = [("variant", C.c_int), ("blocks_per_sm", C.c_int), ("scatterings_per_s", C.c_double),
                ("warps_per_block", C.c_int), ("refill_min", C.c_int)]


class ScatterIO(C.Structure):
    _fields_ = [("x", C.c_double), ("k", C.c_double * 3), ("a", C.c_double), ("g", C.c_double),
                ("atau0", C.c_double), ("phase", C.c_int32), ("pid", C.c_uint64), ("event", C.c_uint32),
                ("x_f", C.c_double), ("k_f", C.c_double * 3), ("u_atom", C.c_double * 3),
                ("u_par", C.c_double), ("x_crit", C.c_double), ("RQ", C.c_double), ("mu", C.c_double),
                ("n_trials", C.c_int32)]


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libcolt.so, building it first when it is missing or stale and nvcc
    is available.  Raises if the library cannot be loaded."""
    global _LIB
    if _LIB is None:
        try:
            if _build.stale():
                _build.build()
        except RuntimeError as e:
            if not os.path.exists(_build.LIB):
                raise ColtError(COLT_ECUDA, f"libcolt.so is missing and cannot be built: {e}")
        if not os.path.exists(_build.LIB):
            raise ColtError(COLT_ECUDA, "libcolt.so is missing")
        L = C.CDLL(_build.LIB)
        P, I, U64, D, SZ = C.c_void_p, C.c_int, C.c_uint64, C.c_double, C.c_size_t
        sig = {
            "colt_init": (I, [C.POINTER(P), I, SZ, P]),
            "colt_finalize": (None, [P]),
            "colt_last_error": (C.c_char_p, [P]),
            "colt_device_info": (I, [P, C.POINTER(I), C.POINTER(SZ), C.POINTER(I), C.POINTER(I)]),
            "colt_create_grid": (I, [P, P, C.POINTER(U64)]),
            "colt_destroy_grid": (I, [P, U64]),
            "colt_read_cells": (I, [P, U64, P, SZ]),
            "colt_run": (I, [P, U64, P, P]),
            "colt_run_batch": (I, [P, I, P, P, P]),
            "colt_solve": (I, [P, P, P, P]),
            "colt_submit": (I, [P, U64, P, C.POINTER(U64)]),
            "colt_submit_many": (I, [P, I, P, P, P]),
            "colt_poll": (I, [P, U64, C.POINTER(I), P]),
            "colt_wait": (I, [P, U64, D]),
            "colt_read_spectrum": (I, [P, U64, I, P, SZ]),
            "colt_read_image": (I, [P, U64, I, P, SZ]),
            "colt_read_result": (I, [P, U64, P]),
            "colt_release": (I, [P, U64]),
            "colt_cancel": (I, [P, U64]),
            "colt_set_launch_config": (I, [P, I, I, P]),
            "colt_voigt": (I, [P, P, P, P, SZ, I, I]),
            "colt_scatter": (I, [P, P, SZ, U64, I]),
            "colt_run_noalloc": (I, [I, P, P, P, P]),
            "colt_autotune": (I, [P, U64, P, P]),
            "colt_set_cell_luminosity": (I, [P, U64, P, I]),
        }
        for name, (rt, args) in sig.items():
            f = getattr(L, name)
            f.restype = rt
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(ctx, rc):
    if rc != COLT_OK:
        msg = lib().colt_last_error(ctx)
        raise ColtError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ context --
def colt_init(device: int = 0, mem_budget_bytes: int = 0, cuda_stream: Optional[int] = None):
    ctx = C.c_void_p()
    rc = lib().colt_init(C.byref(ctx), int(device), int(mem_budget_bytes),
                         C.c_void_p(cuda_stream) if cuda_stream else None)
    if rc != COLT_OK:
        raise ColtError(rc, "colt_init failed (no usable CUDA device?)")
    return ctx


def colt_finalize(ctx):
    lib().colt_finalize(ctx)


def colt_last_error(ctx) -> str:
    m = lib().colt_last_error(ctx)
    return m.decode() if m else ""


def colt_device_info(ctx):
    sm, maj, mnr, l2 = C.c_int(), C.c_int(), C.c_int(), C.c_size_t()
    _check(ctx, lib().colt_device_info(ctx, C.byref(sm), C.byref(l2), C.byref(maj), C.byref(mnr)))
    return dict(sm_count=sm.value, l2_bytes=l2.value, cc=(maj.value, mnr.value))


# -------------------------------------------------------------------- grids --
def grid_desc(grid, f_nl: float = 0.5, device_fields=None):
    """colt_grid_desc for a synth.Grid.  device_fields: optional dict of torch
    CUDA tensors (n_HI, T, vx, vy, vz, k_dust) to pass as device pointers."""
    d = GridDesc()
    keep = []
    d.kind = int(grid.kind)
    d.nx, d.ny, d.nz = [int(v) for v in grid.shape]
    d.lo = (C.c_double * 3)(*[float(v) for v in grid.lo])
    d.hi = (C.c_double * 3)(*[float(v) for v in grid.hi])
    d.periodic_xy = int(bool(grid.periodic_xy))
    d.n_cells = int(grid.n_cells)
    if grid.kind == COLT_OCTREE:
        lv = np.ascontiguousarray(grid.leaf_level, np.uint8)
        ijk = np.ascontiguousarray(grid.leaf_ijk, np.uint32)
        keep += [lv, ijk]
        d.leaf_level, d.leaf_ijk = _ptr(lv), _ptr(ijk)
    names = ["n_HI", "T", "vx", "vy", "vz", "k_dust"]
    if device_fields is not None:
        for nm in names:
            t = device_fields.get(nm)
            setattr(d, nm, t.data_ptr() if t is not None else None)
            keep.append(t)
        d.fields_mem = COLT_MEM_DEVICE
    else:
        for nm in names:
            a = getattr(grid, nm)
            if a is None:
                continue
            a = np.ascontiguousarray(a, np.float32)
            keep.append(a)
            setattr(d, nm, a.ctypes.data)
        d.fields_mem = COLT_MEM_HOST
    d.f_nl = float(f_nl)
    return d, keep


def colt_create_grid(ctx, grid, f_nl: float = 0.5, device_fields=None) -> int:
    """Create the device grid; a synth.Grid carrying cell luminosities
    (grid.lum) also gets them set (colt_set_cell_luminosity)."""
    d, keep = grid_desc(grid, f_nl, device_fields)
    h = C.c_uint64()
    _check(ctx, lib().colt_create_grid(ctx, C.byref(d), C.byref(h)))
    if getattr(grid, "lum", None) is not None:
        try:
            colt_set_cell_luminosity(ctx, h.value, grid.lum)
        except ColtError:
            lib().colt_destroy_grid(ctx, h)
            raise
    return h.value


def colt_set_cell_luminosity(ctx, grid: int, lum):
    """lum: per-cell luminosities, a float64 numpy array (host) or a CUDA
    torch tensor of float64 (device)."""
    if hasattr(lum, "data_ptr"):
        _check(ctx, lib().colt_set_cell_luminosity(ctx, C.c_uint64(grid), C.c_void_p(lum.data_ptr()),
                                                   COLT_MEM_DEVICE))
    else:
        a = np.ascontiguousarray(lum, np.float64)
        _check(ctx, lib().colt_set_cell_luminosity(ctx, C.c_uint64(grid), _ptr(a), COLT_MEM_HOST))


def colt_destroy_grid(ctx, grid: int):
    _check(ctx, lib().colt_destroy_grid(ctx, C.c_uint64(grid)))


def colt_read_cells(ctx, grid: int, n_cells: int) -> np.ndarray:
    out = np.zeros((n_cells, 8), np.float32)
    _check(ctx, lib().colt_read_cells(ctx, C.c_uint64(grid), _ptr(out), out.size))
    return out


# --------------------------------------------------------------------- runs --
def run_params(spec, images: bool = False):
    p = RunParams()
    p.n_packets = int(spec.n_packets)
    p.seed = int(spec.seed)
    p.src_pos = (C.c_double * 3)(*[float(v) for v in spec.src_pos])
    p.src_sigma = float(spec.src_sigma)
    p.core_skip = int(spec.core_skip)
    p.recoil = int(bool(spec.recoil))
    p.phase = int(spec.phase)
    p.tau_esc_max = float(spec.tau_esc_max)
    p.albedo = float(spec.albedo)
    p.max_scatter = int(spec.max_scatter)
    p.spec_units = int(spec.spec_units)
    p.T_ref = float(spec.T_ref)
    p.spec_lo, p.spec_hi, p.spec_nbins = float(spec.spec_lo), float(spec.spec_hi), int(spec.spec_nbins)
    n = len(spec.cameras)
    cams = (Camera * max(n, 1))()
    for i, c in enumerate(spec.cameras):
        cams[i].dir = (C.c_double * 3)(*[float(v) for v in c.direction])
        cams[i].npix = int(c.npix) if images else 0
    p.n_cam = n
    p.cams = C.cast(cams, C.c_void_p)
    p.cam_units = int(spec.cam_units)
    p.cam_lo, p.cam_hi, p.cam_nbins = float(spec.cam_lo), float(spec.cam_hi), int(spec.cam_nbins)
    p.fov_half = float(spec.fov_half)
    p.precision = int(spec.precision)
    p.block_size = 0
    p.blocks_per_sm = int(getattr(spec, "blocks_per_sm", 0) or 0)
    p.pid_offset = int(getattr(spec, "pid_offset", 0) or 0)
    p.emission = int(getattr(spec, "emission", 0) or 0)
    p.source = int(getattr(spec, "source", 0) or 0)
    srcs = list(getattr(spec, "sources", None) or [])
    p.n_sources = len(srcs)
    arr = (Source * max(1, len(srcs)))()
    for i, (pos, sig, w) in enumerate(srcs):
        arr[i].pos = (C.c_double * 3)(*[float(v) for v in pos])
        arr[i].sigma = float(sig)
        arr[i].weight = float(w)
    p.sources = C.cast(arr, C.c_void_p) if srcs else None
    return p, (cams, arr)


def _result_arrays(spec, per_packet, images, grid_npix=None):
    r = Result()
    out = {"spec": np.zeros(spec.spec_nbins, np.uint64)}
    r.spec = out["spec"].ctypes.data
    n = len(spec.cameras)
    if n:
        out["cam_spec"] = np.zeros((n, spec.cam_nbins), np.float64)
        out["cam_spec2"] = np.zeros((n, spec.cam_nbins), np.float64)
        r.cam_spec, r.cam_spec2 = out["cam_spec"].ctypes.data, out["cam_spec2"].ctypes.data
        if images:
            m = sum(int(c.npix) ** 2 for c in spec.cameras) * spec.cam_nbins
            out["cam_image"] = np.zeros(m, np.float64)
            r.cam_image = out["cam_image"].ctypes.data
    if per_packet:
        out["pk_status"] = np.zeros(spec.n_packets, np.int32)
        out["pk_nscat"] = np.zeros(spec.n_packets, np.uint64)
        out["pk_freq"] = np.zeros(spec.n_packets, np.float64)
        r.pk_status, r.pk_nscat, r.pk_freq = (out["pk_status"].ctypes.data, out["pk_nscat"].ctypes.data,
                                              out["pk_freq"].ctypes.data)
    return r, out


def _unpack(r, out):
    for f in ("n_emitted", "n_escaped", "n_absorbed", "n_capped", "n_scat", "n_scat_hi", "n_cell_visits",
              "n_peel_visits", "n_peel_rays", "spec_under", "spec_over", "kernel_ms"):
        out[f] = getattr(r, f)
    return out


def colt_run(ctx, grid: int, spec, per_packet: bool = False, images: bool = False) -> dict:
    p, cams = run_params(spec, images)
    r, out = _result_arrays(spec, per_packet, images)
    _check(ctx, lib().colt_run(ctx, C.c_uint64(grid), C.byref(p), C.byref(r)))
    return _unpack(r, out)


def colt_run_batch(ctx, grids, specs, per_packet: bool = False, images: bool = False, outputs: bool = True):
    """Several solves in one persistent launch.  outputs=False requests only
    the counters (tallies stay on the device and are discarded)."""
    n = len(grids)
    keep = []
    ps = (RunParams * n)()
    rs = (Result * n)()
    outs = []
    for i, (g, sp) in enumerate(zip(grids, specs)):
        p, cams = run_params(sp, images)
        keep.append(cams)
        ps[i] = p
        if outputs:
            r, out = _result_arrays(sp, per_packet, images)
        else:
            r, out = Result(), {}
        rs[i] = r
        outs.append(out)
    hs = (C.c_uint64 * n)(*[int(g) for g in grids])
    _check(ctx, lib().colt_run_batch(ctx, n, hs, ps, rs))
    return [_unpack(rs[i], outs[i]) for i in range(n)]


def colt_solve(ctx, grid, spec, f_nl: float = 0.5, images: bool = False) -> dict:
    """End-to-end call with host fields: grid build + run + result copy."""
    d, keep = grid_desc(grid, f_nl)
    p, cams = run_params(spec, images)
    r, out = _result_arrays(spec, False, images)
    _check(ctx, lib().colt_solve(ctx, C.byref(d), C.byref(p), C.byref(r)))
    return _unpack(r, out)


# ------------------------------------------------------------------ serving --
def colt_autotune(ctx, grid: int, spec) -> dict:
    """Measure and keep the fastest launch configuration for the spec's
    precision and the grid's kind (see colt.h)."""
    p, cams = run_params(spec, False)
    out = LaunchConfig()
    _check(ctx, lib().colt_autotune(ctx, C.c_uint64(grid), C.byref(p), C.byref(out)))
    return dict(variant=out.variant, blocks_per_sm=out.blocks_per_sm, scatterings_per_s=out.scatterings_per_s,
                warps_per_block=out.warps_per_block, refill_min=out.refill_min)


def colt_set_launch_config(ctx, precision: int, kind: int, variant: int = 0, blocks_per_sm: int = 0,
                           warps_per_block: int = 8, refill_min: int = 1):
    c = LaunchConfig(variant=variant, blocks_per_sm=blocks_per_sm, scatterings_per_s=0.0,
                     warps_per_block=warps_per_block, refill_min=refill_min)
    _check(ctx, lib().colt_set_launch_config(ctx, int(precision), int(kind), C.byref(c)))


def colt_submit(ctx, grid: int, spec, images: bool = True) -> int:
    """Queue a solve.  Cameras with npix > 0 tally image cubes unless
    images=False (then only their spectra are tallied)."""
    p, cams = run_params(spec, images)
    h = C.c_uint64()
    _check(ctx, lib().colt_submit(ctx, C.c_uint64(grid), C.byref(p), C.byref(h)))
    return h.value


def colt_submit_many(ctx, reqs, images: bool = True) -> list:
    """Queue several solves at once, reqs = [(grid, spec), ...]: all are
    checked before any is queued, and they are scheduled together."""
    n = len(reqs)
    made = [run_params(spec, images) for _, spec in reqs]   # keeps each camera/source array alive
    ps = (RunParams * max(n, 1))(*[m[0] for m in made])
    gs = (C.c_uint64 * max(n, 1))(*[g for g, _ in reqs])
    hs = (C.c_uint64 * max(n, 1))()
    _check(ctx, lib().colt_submit_many(ctx, C.c_int(n), gs, ps, hs))
    return [hs[i] for i in range(n)]


def colt_poll(ctx, req: int) -> dict:
    done = C.c_int()
    st = Stats()
    _check(ctx, lib().colt_poll(ctx, C.c_uint64(req), C.byref(done), C.byref(st)))
    return dict(done=bool(done.value), admitted=bool(st.admitted), packets_done=st.packets_done,
                packets_total=st.packets_total, latency_ms=st.submit_to_done_ms, launches=st.ctx_launches,
                cancelled=bool(st.cancelled), timed_launches=st.ctx_timed_launches, kernel_ms=st.ctx_kernel_ms,
                longest_history=st.longest_history, cell_visits=st.ctx_cell_visits,
                peel_visits=st.ctx_peel_visits)


def colt_wait(ctx, req: int, timeout_ms: float = -1.0):
    _check(ctx, lib().colt_wait(ctx, C.c_uint64(req), float(timeout_ms)))


def colt_read_spectrum(ctx, req: int, camera: int, nbins: int) -> np.ndarray:
    buf = np.zeros(nbins, np.float64)
    _check(ctx, lib().colt_read_spectrum(ctx, C.c_uint64(req), int(camera), _ptr(buf), nbins))
    return buf


def colt_read_image(ctx, req: int, camera: int, npix: int, nbins: int) -> np.ndarray:
    """Image cube [v][u][bin] of one camera of a finished request."""
    buf = np.zeros((npix, npix, nbins), np.float64)
    _check(ctx, lib().colt_read_image(ctx, C.c_uint64(req), int(camera), _ptr(buf), buf.size))
    return buf


def colt_read_result(ctx, req: int, spec) -> dict:
    r, out = _result_arrays(spec, False, False)
    _check(ctx, lib().colt_read_result(ctx, C.c_uint64(req), C.byref(r)))
    return _unpack(r, out)


def colt_cancel(ctx, req: int):
    _check(ctx, lib().colt_cancel(ctx, C.c_uint64(req)))


def colt_release(ctx, req: int):
    _check(ctx, lib().colt_release(ctx, C.c_uint64(req)))


# ---------------------------------------------------- solve without allocating --
class GridView(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("periodic_xy", C.c_int), ("records", C.c_void_p)]


class DeviceTallies(C.Structure):
    _fields_ = [("spec", C.c_void_p), ("counters", C.c_void_p), ("cam_spec", C.c_void_p),
                ("cam_spec2", C.c_void_p), ("cam_image", C.c_void_p)]


def _noalloc_layout(name, t, dtype, numel):
    """The C entry point takes bare device pointers and no lengths, so every
    buffer is checked here: a wrong size, type or layout would make the
    kernel read or write outside it."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name}: {t.numel()} elements, expected {numel}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: not contiguous")


def _noalloc_device(name, t):
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name}: not a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is cuda:{torch.cuda.current_device()}")


def check_noalloc_args(grids, records, specs, tallies, images=False):
    """Raise ValueError unless every records and tally tensor has the type,
    layout and length colt_run_noalloc will access (all checked first) and
    lies on the current CUDA device."""
    import torch
    n = len(grids)
    if not (len(records) == len(specs) == len(tallies) == n):
        raise ValueError("grids, records, specs and tallies must have the same length")
    checked = []
    for i, (g, rec, sp, t) in enumerate(zip(grids, records, specs, tallies)):
        nx, ny, nz = [int(v) for v in g.shape]
        want = [(f"records[{i}]", rec, torch.float32, nx * ny * nz * 8),
                (f"tallies[{i}]['spec']", t.get("spec"), torch.int64, int(sp.spec_nbins)),
                (f"tallies[{i}]['counters']", t.get("counters"), torch.int64, 8)]
        ncam = len(sp.cameras)
        if ncam:
            want += [(f"tallies[{i}]['{f}']", t.get(f), torch.float64, ncam * int(sp.cam_nbins))
                     for f in ("cam_spec", "cam_spec2")]
            npx = sum(int(c.npix) ** 2 for c in sp.cameras) if images else 0
            if npx:
                want.append((f"tallies[{i}]['cam_image']", t.get("cam_image"), torch.float64,
                             npx * int(sp.cam_nbins)))
        for name, tensor, dtype, numel in want:
            _noalloc_layout(name, tensor, dtype, numel)
            checked.append((name, tensor))
    for name, tensor in checked:
        _noalloc_device(name, tensor)


def colt_run_noalloc(grids, records, specs, tallies, cuda_stream=None, images=False):
    """Blocking solve(s) without device allocation.  grids: synth.Grid list
    (geometry only); records: device tensors (8 floats per cell); tallies:
    dicts of device tensors spec, counters, cam_spec, cam_spec2, cam_image.
    Every tensor is checked (ValueError) before the call.  Returns the C status
    code (0 = COLT_OK)."""
    check_noalloc_args(grids, records, specs, tallies, images)
    n = len(grids)
    gv = (GridView * n)()
    ps = (RunParams * n)()
    ts = (DeviceTallies * n)()
    keep = []
    for i, (g, rec, sp, t) in enumerate(zip(grids, records, specs, tallies)):
        gv[i].nx, gv[i].ny, gv[i].nz = [int(v) for v in g.shape]
        gv[i].lo = (C.c_double * 3)(*[float(v) for v in g.lo])
        gv[i].hi = (C.c_double * 3)(*[float(v) for v in g.hi])
        gv[i].periodic_xy = int(bool(g.periodic_xy))
        gv[i].records = rec.data_ptr()
        p, cams = run_params(sp, images)
        keep.append(cams)
        ps[i] = p
        for f in ("spec", "counters", "cam_spec", "cam_spec2", "cam_image"):
            v = t.get(f)
            setattr(ts[i], f, v.data_ptr() if v is not None else None)
    return lib().colt_run_noalloc(n, gv, ps, ts, C.c_void_p(cuda_stream) if cuda_stream else None)


# ------------------------------------------------------------------- parity --
def colt_voigt(ctx, a, x, precision: int = COLT_MIXED) -> np.ndarray:
    dt = np.float64 if precision == COLT_PLAIN else np.float32
    a = np.ascontiguousarray(a, dt)
    x = np.ascontiguousarray(x, dt)
    H = np.empty_like(a)
    _check(ctx, lib().colt_voigt(ctx, _ptr(a), _ptr(x), _ptr(H), a.size, int(precision), COLT_MEM_HOST))
    return H


SCATTER_OUT = ("x_f", "k_f", "u_atom", "u_par", "x_crit", "RQ", "mu", "n_trials")


def colt_scatter(ctx, inp: dict, seed: int, precision: int = COLT_MIXED) -> dict:
    n = len(inp["x"])
    arr = (ScatterIO * n)()
    v = np.ctypeslib.as_array(arr)
    v["x"] = inp["x"]
    v["k"] = np.asarray(inp["k"]).reshape(n, 3)
    v["a"] = inp["a"]
    v["g"] = inp["g"]
    v["atau0"] = inp["atau0"]
    v["phase"] = inp["phase"]
    v["pid"] = inp["pid"]
    v["event"] = inp["event"]
    _check(ctx, lib().colt_scatter(ctx, C.cast(arr, C.c_void_p), n, int(seed), int(precision)))
    return {f: np.array(v[f]) for f in SCATTER_OUT}
