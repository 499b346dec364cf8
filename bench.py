"""Benchmark of the Lyman-alpha packet transport on one (or N) GB300.

Default run (`python bench.py [--gpus N --steps K --warmup W]`) prints ONE
JSON line.  Its headline (value, e2e, roofline, cpu_baseline, clocks) is the
largest workload:

cosmo     the synthetic cosmological box (1 Mpc^3 comoving at z = 10,
          lognormal density on an octree of 9.4e6 leaves, levels 7-12), five
          sources at the highest density peaks, peel-off to three cameras of
          512^2 pixels x 256 bins over +-1000 km/s, mixed precision.  A step is
          one solve per source of --cosmo-packets packets (disjoint packet ids
          per step and rank).  The K timed steps are submitted together to the
          serving scheduler (colt_submit_many), as a user submits a job of
          many steps: they share persistent launches, so one step's longest
          histories run beside the other steps' work.  value = scatterings/s (executed,
          core-skipped ones not counted) over the device-timed region (CUDA
          events on the library's stream, grid resident); photons/s and served
          p50/p99 beside it.  The same pass gives e2e: the grid built from host
          fields, the K steps, and every solve's spectra and image cubes read
          back to the host.  Warm-up steps run the same solves with histories
          capped at 1e4 scatterings.

Secondary workloads, each with its own clocks (rank 0, N = 1), under
"workloads":
sphere128 the 128^3 dusty-sphere suite (tau0 {1e5,1e6,1e7} x v_max {-200,0,200}
          km/s, dust tau 1, A = 0.32, six 128^2 x 200 cameras): served steps of
          nine solves; the plain single-launch kernel on the whole job (1e6
          packets per case in one launch); the plain FP64 kernel on one solve
          (tau0 = 1e5 static, --fp64-packets)
halo      the synthetic octree AMR halo (2.05e6 leaves, levels 6-12), central
          Gaussian source of 0.1 kpc, six 128^2 x 200 cameras: served steps
serving   256 requests (spheres or slabs on 64^3, tau0, T, v_max, dust and
          packet counts drawn per request, seeds 4000 + i) arriving as a
          Poisson process at 75% of the throughput measured on the same mix
          submitted at once; p50/p99 latency and throughput

--impl reference  the FP64 CPU oracle on the host cores, bounded samples of the
                  headline workload (one source's packets per step, cycling)
--workload W      one workload alone (sphere128, halo, halo_diffuse, cosmo,
                  serving, tslab, galaxies), for profiling
--single-case I   one blocking solve of sphere-suite case I (profiling driver)
--profile-case W  one short capped solve of workload W (ncu capture driver);
          --profile-no-cameras: the same solves without cameras
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1409_4480_gb300 import synth as S  # noqa: E402

TAU0S = (1e5, 1e6, 1e7)
VMAX = (-200.0, 0.0, 200.0)
PACKETS_PER_CASE_JOB = 10 ** 6
METRIC = "scatterings/s & photons/s at oracle-matched spectra; served p50/p99 latency"
UNIT = "scatterings/s"
WORKLOAD = "sphere128_T1e4_dust1_9cases_6cam"


def cases():
    return [(t, v) for t in TAU0S for v in VMAX]


def case_grid(tau0, v, n=128):
    return S.sphere(n, 1e4, tau0, v_max_kms=v, tau_dust=1.0)


def case_spec(i, n_packets, pid_offset, images=True):
    return S.RunSpec(n_packets=n_packets, seed=200 + i, albedo=0.32, spec_units=1, spec_lo=-1000.0,
                     spec_hi=1000.0, spec_nbins=200, cameras=S.axis_cameras(128 if images else 0),
                     cam_units=1, cam_lo=-1000.0, cam_hi=1000.0, cam_nbins=200, precision=1,
                     pid_offset=pid_offset)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = ("paper_1409_4480_gb300/csrc/transport.cu", "paper_1409_4480_gb300/csrc/device.cuh",
                  "paper_1409_4480_gb300/csrc/internal.h", "paper_1409_4480_gb300/csrc/octree.cuh",
                  "paper_1409_4480_gb300/csrc/cellpos.cuh")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------- oracle legs --
def oracle_sample(target_s=15.0, case=(1e6, 0.0), cores=0):
    """Time the FP64 oracle, as it stands, on a bounded sample of one case."""
    import oracle as O
    g = case_grid(*case)
    i = cases().index(case)
    n = 16
    O.run(g, case_spec(i, 4, 0, images=False), n_threads=cores)  # warm (page-in, grid derivation)
    while True:
        r = O.run(g, case_spec(i, n, 0, images=False), n_threads=cores)
        if r["transport_seconds"] > target_s / 4 or n >= 1 << 20:
            break
        n *= 4
    if r["transport_seconds"] < target_s:
        n = int(n * target_s / max(r["transport_seconds"], 1e-3))
        r = O.run(g, case_spec(i, n, 0, images=False), n_threads=cores)
    t = r["transport_seconds"]
    return dict(value=r["n_scat"] / t, unit=UNIT, cores=r["n_threads"],
                photons_per_s=n / t, seconds=t,
                sample=f"{n} packets of the tau0={case[0]:g}, v_max={case[1]:g} km/s case (6 cameras x 200 "
                       f"bins peel-off, no images); the packet loop timed, grid derivation excluded as on the GPU")


def run_reference(args):
    """The FP64 oracle, as it stands, on the host cores: each step a bounded
    sample of the headline workload (--ref-packets packets of one source,
    cycling through the five; camera spectra, no images), the grid derived
    once; the packet loops timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    g, srcs, cams, cnb, label = octree_workload("cosmo")
    cams0 = [S.Camera(c.direction, 0) for c in cams]
    n = args.ref_packets
    specs = []
    for st in range(args.warmup + args.steps):
        j = st % len(srcs)
        specs.append(cosmo_specs(srcs[j:j + 1], cams0, cnb, n, 10 ** 9 + st * n)[0])
        specs[-1].seed = 300 + j
    rs = O.run_many(g, specs, workers=1)
    timed = rs[args.warmup:]
    t_all = sum(r["transport_seconds"] for r in timed)
    n_scat = sum(r["n_scat"] for r in timed)
    value = n_scat / t_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "photons_per_s": n * args.steps / t_all,
            "config": {"workload": label, "packets_per_step": n, "sources": "one per step, cycling through the five",
                       "cameras": "3 camera spectra x 256 bins (no images)", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n} packets per step of one source of {label}, cycling through the five "
                                       f"sources; the packet loop timed on all host cores, grid derivation "
                                       f"excluded as on the GPU"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg --
def run_single_case(args):
    from paper_1409_4480_gb300 import colt as C
    ctx = C.colt_init(0)
    t, v = cases()[args.single_case]
    h = C.colt_create_grid(ctx, case_grid(t, v))
    sp = case_spec(args.single_case, args.packets_per_case, 0, images=not args.no_images)
    if args.max_scatter > 0:
        sp.max_scatter = args.max_scatter      # bounded histories: steady-state profiles
    r = C.colt_run(ctx, h, sp)
    print(json.dumps({"case": args.single_case, "packets": args.packets_per_case, "kernel_ms": r["kernel_ms"],
                      "scatterings": r["n_scat"], "peel_visits": r["n_peel_visits"],
                      "cell_visits": r["n_cell_visits"]}))
    C.colt_finalize(ctx)


def run_gpu(args):
    import torch
    from paper_1409_4480_gb300 import colt as C

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = C.colt_init(local, 0, stream.cuda_stream)
    info = C.colt_device_info(ctx)
    B = args.packets_per_case
    img = not args.no_images
    grids_h = [case_grid(t, v) for t, v in cases()]
    hs = [C.colt_create_grid(ctx, g) for g in grids_h]
    # launch configuration measured on the static tau0 = 1e6 case (before warm-up)
    tuned = C.colt_autotune(ctx, hs[4], case_spec(4, B, 0, images=False))

    def specs_of(s):
        off = (s * world + rank) * B          # disjoint packet ids per (step, rank)
        return [case_spec(i, B, off, images=img) for i in range(9)]

    def submit(s):
        return [(C.colt_submit(ctx, hs[i], sp), sp) for i, sp in enumerate(specs_of(s))]

    def finish(reqs):
        out = []
        for rid, sp in reqs:
            C.colt_wait(ctx, rid, -1.0)
        for rid, sp in reqs:
            st = C.colt_poll(ctx, rid)
            res = C.colt_read_result(ctx, rid, S.RunSpec(**{**sp.__dict__, "cameras": []}))
            out.append((st, res))
            C.colt_release(ctx, rid)
        return out

    for s in range(args.warmup):
        finish(submit(s))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = launch_count(C, ctx, hs[0])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        t0 = time.perf_counter()
        reqs = []
        for s in range(args.warmup, args.warmup + args.steps):
            reqs += submit(s)
        done = finish(reqs)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1)
    launches = launch_count(C, ctx, hs[0]) - launches0
    tot_scat = sum(r["n_scat"] for _, r in done)
    tot_pk = sum(r["n_emitted"] for _, r in done)
    lat = [st["latency_ms"] for st, _ in done]
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        c = torch.tensor([tot_scat, tot_pk], device="cuda", dtype=torch.float64)
        dist.all_reduce(c)
        tot_scat, tot_pk = int(c[0].item()), int(c[1].item())
    value = tot_scat / (ms / 1e3)
    photons = tot_pk / (ms / 1e3)

    # plain: the blocking single-launch call on one step (visit counts for the roofline)
    s_plain = args.warmup + args.steps
    tp0 = time.perf_counter()
    res_plain = C.colt_run_batch(ctx, hs, specs_of(s_plain), images=img, outputs=False)
    plain_wall = time.perf_counter() - tp0
    plain_scat = sum(r["n_scat"] for r in res_plain)
    plain_ms = res_plain[0]["kernel_ms"]
    visits = (res_plain[0]["n_cell_visits"], res_plain[0]["n_peel_visits"], res_plain[0]["n_peel_rays"])

    # end to end: host fields -> grids -> served solves -> results (spectra + images) on the host,
    # over as many steps as the device-timed value (each step uploads its own grids and reads its
    # own results back); a failure there falls back to one step
    e2e = None
    if not args.no_e2e:
        s_e2e = s_plain + 1

        def e2e_leg(n_steps):
            h2d = d2h = 0
            scat = 0
            made, rids = [], []
            ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev2.record(stream)
            try:
                steps = []
                for s in range(n_steps):
                    ghs = []
                    for g in grids_h:
                        ghs.append(C.colt_create_grid(ctx, g))
                        made.append(ghs[-1])        # released in `finally` if a later call fails
                    h2d += sum(6 * 4 * g.n_cells for g in grids_h)
                    steps.append(ghs)
                for s, ghs in enumerate(steps):
                    off = ((s_e2e + s) * world + rank) * B
                    for i, gh in enumerate(ghs):
                        sp = case_spec(i, B, off, images=img)
                        rids.append((C.colt_submit(ctx, gh, sp), sp))
                for rid, sp in rids:
                    C.colt_wait(ctx, rid, -1.0)
                while rids:
                    rid, sp = rids.pop(0)
                    r = C.colt_read_result(ctx, rid, sp) if not img else read_with_images(C, ctx, rid, sp)
                    scat += r["n_scat"]
                    d2h += sum(v.nbytes for k, v in r.items() if isinstance(v, np.ndarray))
                    C.colt_release(ctx, rid)
                for gh in made:
                    C.colt_destroy_grid(ctx, gh)
                made = []
                ev3.record(stream)
                torch.cuda.synchronize()
            finally:
                for rid, sp in rids:
                    try:
                        C.colt_wait(ctx, rid, -1.0)
                        C.colt_release(ctx, rid)
                    except C.ColtError:
                        pass
                for gh in made:
                    try:
                        C.colt_destroy_grid(ctx, gh)
                    except C.ColtError:
                        pass
            e_ms = ev2.elapsed_time(ev3)
            return {"value": scat / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d // n_steps,
                    "d2h_bytes_per_step": d2h // n_steps, "ms_per_step": e_ms / n_steps, "steps": n_steps,
                    "path": "colt_create_grid (host fields) -> colt_submit -> colt_wait -> colt_read_result "
                            "(escape + camera spectra + image cubes) -> colt_destroy_grid, every step"}

        try:
            e2e = e2e_leg(args.steps)
        except Exception as exc:          # noqa: BLE001 -- report, then measure one step
            e2e = e2e_leg(1)
            e2e["note"] = f"{args.steps}-step leg failed ({type(exc).__name__}); one step measured"

    rf = roofline(profile_units("sphere128"), plain_scat, plain_ms, value, info)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(args.cpu_seconds)
        cpu["kind"] = "oracle"
    lat_sorted = sorted(lat)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "photons_per_s": photons,
            "served_latency_ms": {"p50": float(np.percentile(lat_sorted, 50)),
                                  "p99": float(np.percentile(lat_sorted, 99)), "n_requests": len(lat),
                                  "arrivals": "burst: all steps' requests submitted at t0"},
            "plain": {"value": plain_scat / (plain_ms / 1e3), "unit": UNIT, "kernel_ms": plain_ms,
                      "wall_s": plain_wall, "path": "colt_run_batch, one blocking launch of the 9 solves",
                      "cell_visits_per_s": visits[0] / (plain_ms / 1e3),
                      "peel_visits_per_s": visits[1] / (plain_ms / 1e3),
                      "record_bytes_per_visit": 32},
            "config": {"workload": WORKLOAD,
                       "cases": "tau0 {1e5,1e6,1e7} x v_max {-200,0,200} km/s, tau_d=1, A=0.32",
                       "packets_per_case_per_step": B, "steps_per_job": PACKETS_PER_CASE_JOB // B,
                       "cameras": "6 x 128^2 x 200" if img else "6 x 200 (no images)",
                       "grid": "128^3 Cartesian, 32 B records", "precision": "mixed (FP32 transport, FP64 tau/escape)",
                       "launch": "served: colt_submit of 9 solves per step, persistent launches in flight",
                       "launch_config": {"variant": tuned["variant"], "blocks_per_sm": tuned["blocks_per_sm"],
                                         "source": "colt_autotune on the tau0=1e6 static case"},
                       "l2": "records 9 x 67 MB + tallies 9 x 157 MB per step > 129 MB L2: inputs larger than L2"},
            "gpu_launches": launches,
            "counts": {"scatterings": tot_scat, "packets": tot_pk,
                       "plain_step": {"scatterings": plain_scat, "cell_visits": visits[0], "peel_visits": visits[1],
                                      "peel_rays": visits[2]}},
            "roofline": rf,
            "clocks": clk.summary(), "wall_s": wall}
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    C.colt_finalize(ctx)
    if dist:
        dist.destroy_process_group()


def _rank_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def octree_workload(name):
    """(grid, list of (source position, source sigma), cameras, camera bins, label)"""
    if name == "halo":
        g = S.halo()
        return g, [((0.0, 0.0, 0.0), 100.0 * S.PC_CM)], S.axis_cameras(128), 200, \
            f"halo_octree_{g.n_cells}leaves_6cam"
    if name == "halo_diffuse":
        # the same halo emitting from its gas (recombination + collisional
        # excitation per leaf): one diffuse source
        g = S.halo(emission=True)
        return g, [None], S.axis_cameras(128), 200, f"halo_octree_{g.n_cells}leaves_diffuse_6cam"
    g, src = S.cosmo_box()
    return g, [(p, 0.0) for p in src], S.axis_cameras(512, ("+x", "+y", "+z")), 256, \
        f"cosmo_octree_{g.n_cells}leaves_5src_3cam"


def run_octree(args):
    """Served steps on an octree workload (same timing rules as the sphere suite)."""
    import torch
    from paper_1409_4480_gb300 import colt as C
    world, rank, local = _rank_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = C.colt_init(local, 0, stream.cuda_stream)
    g, srcs, cams, cnb, label = octree_workload(args.workload)
    h = C.colt_create_grid(ctx, g)
    B = args.packets_per_case

    def specs_of(s):
        out = []
        for j, src in enumerate(srcs):
            off = ((s * world + rank) * len(srcs) + j) * B
            pos, sig = src if src is not None else ((0.0, 0.0, 0.0), 0.0)
            out.append(S.RunSpec(n_packets=B, seed=300 + j, src_pos=pos, src_sigma=sig, albedo=0.32,
                                 spec_units=1, spec_lo=-1000.0, spec_hi=1000.0, spec_nbins=200, cameras=cams,
                                 cam_units=1, cam_lo=-1000.0, cam_hi=1000.0, cam_nbins=cnb, precision=1,
                                 pid_offset=off, source=0 if src is not None else 1,
                                 core_skip=args.core_skip))
        return out

    def run_steps(s0, n):
        rids = [(C.colt_submit(ctx, h, sp), sp) for s in range(s0, s0 + n) for sp in specs_of(s)]
        res = []
        for rid, sp in rids:
            C.colt_wait(ctx, rid, -1.0)
        for rid, sp in rids:
            st = C.colt_poll(ctx, rid)
            res.append((st, C.colt_read_result(ctx, rid, S.RunSpec(**{**sp.__dict__, "cameras": []}))))
            C.colt_release(ctx, rid)
        return res

    run_steps(0, args.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        done = run_steps(args.warmup, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    scat = sum(r["n_scat"] for _, r in done)
    pk = sum(r["n_emitted"] for _, r in done)
    lat = sorted(st["latency_ms"] for st, _ in done)
    line = {"metric": METRIC, "value": scat / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "photons_per_s": pk / (ms / 1e3),
            "served_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                  "n_requests": len(lat)},
            "config": {"workload": label, "packets_per_source_per_step": B, "sources": len(srcs),
                       "core_skip": ["off", "cell + non-local a tau", "Jeans a tau"][args.core_skip],
                       "grid": f"octree, {g.n_cells} leaves, levels {int(g.leaf_level.min())}-{int(g.leaf_level.max())}",
                       "precision": "mixed (FP32 transport, FP32-pair position and tau, FP64 escape)",
                       "l2": "records + tallies exceed the 129 MB L2"},
            "counts": {"scatterings": scat, "packets": pk}, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    C.colt_finalize(ctx)


def slab_suite():
    """The temperature suites of uniform slabs (App. "Thermal effects"): tau0 = 1e7
    at T = 10, 1e2, 1e3, 1e4, 1e5 K, and a fixed column N_H = 1.7e20 cm^-2
    (tau0 = 1e7 T4^-1/2) at T = 10, 1e2, 1e3, 1e4 K; 64^3 periodic slabs, recoil on,
    angle-averaged spectra over +-300 km/s."""
    out = [("tau0", T, 1e7) for T in (10.0, 1e2, 1e3, 1e4, 1e5)]
    out += [("column", T, 1e7 * (T / 1e4) ** -0.5) for T in (10.0, 1e2, 1e3, 1e4)]
    return out


def run_slab_suite(args):
    """Served steps of the nine temperature-suite slabs (same timing rules)."""
    import torch
    from paper_1409_4480_gb300 import colt as C
    world, rank, local = _rank_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = C.colt_init(local, 0, stream.cuda_stream)
    suite = slab_suite()
    hs = [C.colt_create_grid(ctx, S.slab(64, T, tau0)) for _, T, tau0 in suite]
    B = args.packets_per_case

    def specs_of(s):
        off = (s * world + rank) * B
        return [S.RunSpec(n_packets=B, seed=500 + i, T_ref=T, spec_units=1, spec_lo=-300.0, spec_hi=300.0,
                          spec_nbins=120, precision=1, pid_offset=off) for i, (_, T, _) in enumerate(suite)]

    def run_steps(s0, n):
        rids = [(C.colt_submit(ctx, hs[i], sp), sp) for s in range(s0, s0 + n) for i, sp in enumerate(specs_of(s))]
        res = []
        for rid, sp in rids:
            C.colt_wait(ctx, rid, -1.0)
        for rid, sp in rids:
            res.append((C.colt_poll(ctx, rid), C.colt_read_result(ctx, rid, sp)))
            C.colt_release(ctx, rid)
        return res

    run_steps(0, args.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        done = run_steps(args.warmup, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    scat = sum(r["n_scat"] for _, r in done)
    pk = sum(r["n_emitted"] for _, r in done)
    lat = sorted(st["latency_ms"] for st, _ in done)
    line = {"metric": METRIC, "value": scat / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "photons_per_s": pk / (ms / 1e3),
            "served_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                  "n_requests": len(lat)},
            "config": {"workload": "slab64_temperature_suites_9", "cases": [f"{k} T={T:g} tau0={t:.3g}"
                                                                           for k, T, t in suite],
                       "packets_per_case_per_step": B, "precision": "mixed", "recoil": True},
            "counts": {"scatterings": scat, "packets": pk}, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    C.colt_finalize(ctx)


GALAXY_MODELS = [(m, M) for M in (1e5, 1e6, 1e7, 1e8) for m in ("SE", "SL", "WE", "WL")]


def galaxy_observables(res):
    """Table-3 quantities of one solve: F/F_Omega face-on (+-z cameras) and
    edge-on (+-x, +-y), and the red/blue flux ratios F_r/F_b (Delta v > 0 vs
    < 0) along z, xy and angle-averaged (the escape spectrum)."""
    cs = np.asarray(res["cam_spec"], np.float64)           # cameras: +x -x +y -y +z -z
    ct = cs.sum(axis=1)
    esc = max(float(np.sum(res["spec"])), 1.0)               # the same (wide) velocity range
    h = cs.shape[1] // 2
    rb = lambda s: float(s[h:].sum() / max(s[:h].sum(), 1e-300))
    sp = np.asarray(res["spec"], np.float64)
    return {"F/F_Omega_z": float(ct[4:6].mean() / esc), "F/F_Omega_xy": float(ct[0:4].mean() / esc),
            "Fr/Fb_z": rb(cs[4:6].sum(axis=0)), "Fr/Fb_xy": rb(cs[0:4].sum(axis=0)),
            "Fr/Fb_Omega": float(sp[len(sp) // 2:].sum() / max(sp[:len(sp) // 2].sum(), 1)),
            "f_esc": res["n_escaped"] / max(res["n_emitted"], 1)}


def run_galaxies(args):
    """Served steps over the 16 idealized first-galaxy models (Sec. 5.1:
    SE/SL/WE/WL x M_H,tot = 1e5..1e8 Msun), with their Table-3 observables."""
    import torch
    from paper_1409_4480_gb300 import colt as C
    world, rank, local = _rank_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = C.colt_init(local, 0, stream.cuda_stream)
    grids = [S.galaxy(m, M) for m, M in GALAXY_MODELS]
    hs = [C.colt_create_grid(ctx, g) for g in grids]
    B = args.packets_per_case
    cams = S.axis_cameras(0)

    def specs_of(s):
        off = (s * world + rank) * B
        return [S.RunSpec(n_packets=B, seed=600 + i, recoil=True, albedo=0.0, core_skip=args.core_skip,
                          spec_units=1, spec_lo=-3000.0,
                          spec_hi=3000.0, spec_nbins=300, cameras=cams, cam_units=1, cam_lo=-3000.0,
                          cam_hi=3000.0, cam_nbins=300, precision=1, pid_offset=off)
                for i in range(len(hs))]

    def run_steps(s0, n):
        rids = [(i, C.colt_submit(ctx, hs[i], sp), sp) for s in range(s0, s0 + n)
                for i, sp in enumerate(specs_of(s))]
        res = []
        for i, rid, sp in rids:
            C.colt_wait(ctx, rid, -1.0)
        for i, rid, sp in rids:
            res.append((i, C.colt_poll(ctx, rid), C.colt_read_result(ctx, rid, sp)))
            C.colt_release(ctx, rid)
        return res

    run_steps(0, args.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        done = run_steps(args.warmup, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    scat = sum(r["n_scat"] for _, _, r in done)
    pk = sum(r["n_emitted"] for _, _, r in done)
    lat = sorted(st["latency_ms"] for _, st, _ in done)
    # observables per model, summed over the timed steps
    obs = {}
    for i, (m, M) in enumerate(GALAXY_MODELS):
        rs = [r for j, _, r in done if j == i]
        tot = {k: (np.sum([r[k] for r in rs], axis=0) if k in ("cam_spec", "spec")
                   else sum(r[k] for r in rs)) for k in ("cam_spec", "spec", "n_escaped", "n_emitted")}
        obs[f"{m}{int(round(np.log10(M)))}"] = {k: round(v, 3) for k, v in galaxy_observables(tot).items()}
    line = {"metric": METRIC, "value": scat / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "photons_per_s": pk / (ms / 1e3),
            "served_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                  "n_requests": len(lat)},
            "config": {"workload": "idealized_galaxies_16", "models": "SE/SL/WE/WL x M_H,tot 1e5-1e8 Msun",
                       "core_skip": ["off", "cell + non-local a tau", "Jeans a tau"][args.core_skip],
                       "leaves": [int(g.n_cells) for g in grids], "packets_per_model_per_step": B,
                       "precision": "mixed"},
            "counts": {"scatterings": scat, "packets": pk}, "clocks": clk.summary(), "observables": obs}
    if rank == 0:
        print(json.dumps(line), flush=True)
    C.colt_finalize(ctx)


def serving_requests(n):
    """The serving mix: request i (seed 4000 + i) is a sphere or a slab on a
    64^3 grid with tau0 log-uniform in [1e4, 1e8], T log-uniform in [10, 1e5] K,
    v_max uniform in [-300, 300] km/s, dust tau_d uniform in [0, 2] (A = 0.32)
    and a packet count log-uniform in [1e4, 1e6]; its spectrum has 200 bins over
    +-(6 x_p + u_max) v_th with x_p = 0.93 (a tau0)^(1/3)."""
    out = []
    for i in range(n):
        r = np.random.default_rng(4000 + i)
        geom = "sphere" if r.uniform() < 0.5 else "slab"
        tau0 = float(np.exp(r.uniform(np.log(1e4), np.log(1e8))))
        T = float(np.exp(r.uniform(np.log(10.0), np.log(1e5))))
        v = float(r.uniform(-300.0, 300.0))
        td = float(r.uniform(0.0, 2.0))
        npk = int(np.exp(r.uniform(np.log(1e4), np.log(1e6))))
        vth = 12.85 * np.sqrt(T / 1e4)
        a = 4.702e-4 / np.sqrt(T / 1e4)
        xp = 0.93 * (a * tau0) ** (1.0 / 3.0)
        w = (6.0 * xp + abs(v) / vth) * vth
        out.append(dict(geom=geom, tau0=tau0, T=T, v=v, td=td, n=npk, w=w, seed=4000 + i))
    return out


def serving_grid(q):
    """The 64^3 sphere or slab of one serving-mix request."""
    if q["geom"] == "sphere":
        return S.sphere(64, q["T"], q["tau0"], v_max_kms=q["v"], tau_dust=q["td"])
    return S.slab(64, q["T"], q["tau0"], v_max_kms=q["v"], tau_dust=q["td"])


def run_serving(args):
    """Poisson arrivals into the continuous-batching scheduler."""
    import torch
    from paper_1409_4480_gb300 import colt as C
    world, rank, local = _rank_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = C.colt_init(local, 0, stream.cuda_stream)
    reqs = serving_requests(args.requests)
    grids = [C.colt_create_grid(ctx, serving_grid(q)) for q in reqs]
    specs = [S.RunSpec(n_packets=q["n"], seed=q["seed"], albedo=0.32, spec_units=1, spec_lo=-q["w"], spec_hi=q["w"],
                       spec_nbins=200, precision=1, pid_offset=rank * q["n"]) for q in reqs]

    def drain(rids):
        out = []
        for rid in rids:
            C.colt_wait(ctx, rid, -1.0)
        for rid, sp in zip(rids, specs):
            st = C.colt_poll(ctx, rid)
            r = C.colt_read_result(ctx, rid, sp)
            out.append((st, r))
            C.colt_release(ctx, rid)
        return out

    # calibration: the whole mix submitted at once (also the warm-up)
    t0 = time.perf_counter()
    cal = drain([C.colt_submit(ctx, grids[i], specs[i]) for i in range(len(reqs))])
    t_batch = time.perf_counter() - t0
    rate = args.load * len(reqs) / t_batch              # requests per second
    arr = np.cumsum(np.random.default_rng(4).exponential(1.0 / rate, len(reqs)))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        t0 = time.perf_counter()
        rids = []
        for i in range(len(reqs)):
            while time.perf_counter() - t0 < arr[i]:
                for rid in rids[-8:]:
                    C.colt_poll(ctx, rid)          # drive the scheduler between arrivals
                time.sleep(0.0005)
            rids.append(C.colt_submit(ctx, grids[i], specs[i]))
        done = drain(rids)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    scat = sum(r["n_scat"] for _, r in done)
    pk = sum(r["n_emitted"] for _, r in done)
    lat = np.array([st["latency_ms"] for st, _ in done])
    same = all(np.array_equal(a["spec"], b["spec"]) for (_, a), (_, b) in zip(cal, done))
    line = {"metric": METRIC, "value": scat / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic", "photons_per_s": pk / (ms / 1e3),
            "served_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                  "n_requests": len(lat), "arrivals": f"Poisson, {rate:.3f} requests/s = "
                                  f"{args.load:.2f} x the all-at-once throughput ({len(reqs)} requests in "
                                  f"{t_batch:.1f} s)"},
            "batch_all_at_once": {"wall_s": t_batch, "scatterings_per_s": sum(r["n_scat"] for _, r in cal) / t_batch},
            "results_identical_across_mixes": same,
            "config": {"workload": f"serving_mix_{len(reqs)}req_64cubed", "grids": "64^3 sphere or slab per request",
                       "precision": "mixed", "admission": "memory budget (90% of free HBM)"},
            "counts": {"scatterings": scat, "packets": pk}, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    C.colt_finalize(ctx)


def launch_stats(C, ctx, h=None):
    """(transport launches issued, launches finished and timed, their summed
    CUDA-event milliseconds, their flight cell visits, their peel-off cell
    visits) so far, read through a zero-packet request (it
    completes at once and launches nothing) on grid h, or on a one-cell grid
    made for the purpose."""
    tmp = None
    if h is None:
        tmp = h = C.colt_create_grid(ctx, S.uniform_box((1, 1, 1), (-1.0,) * 3, (1.0,) * 3, 0.0, 1e4))
    rid = C.colt_submit(ctx, h, S.RunSpec(n_packets=0, seed=0))
    st = C.colt_poll(ctx, rid)
    C.colt_release(ctx, rid)
    if tmp is not None:
        C.colt_destroy_grid(ctx, tmp)
    return st["launches"], st["timed_launches"], st["kernel_ms"], st["cell_visits"], st["peel_visits"]


def launch_count(C, ctx, h=None):
    return launch_stats(C, ctx, h)[0]


def read_with_images(C, ctx, rid, sp):
    """colt_read_result with the image cubes requested as well."""
    import ctypes
    r, out = C._result_arrays(sp, False, True)
    C._check(ctx, C.lib().colt_read_result(ctx, ctypes.c_uint64(rid), ctypes.byref(r)))
    return C._unpack(r, out)


# ------------------------------------------------------------------ suite --
PROFILES = os.path.join(ROOT, "profiles")


def kernel_source_hash():
    """sha256 of the transport kernel's sources (a profile is current when it
    names this hash)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_units(name):
    """Per-scattering figures of the transport kernel on workload `name` from
    its committed ncu summary (profiles/k_transport_<name>.md): FP32
    operations (thread-level, FMA = 2) and DRAM bytes per executed
    scattering, and the summary's file name; None when the summary is missing
    or was taken on other kernel sources."""
    import re
    path = os.path.join(PROFILES, f"k_transport_{name}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256: `([0-9a-f]+)`", text)
    if not m_hash or m_hash.group(1) != kernel_source_hash():
        return None
    out = {"profile": os.path.relpath(path, ROOT)}
    for key in ("fp32_flop_per_scattering", "dram_bytes_per_scattering"):
        m = re.search(key + r": ([0-9.eE+-]+)", text)
        out[key] = float(m.group(1)) if m else None
    # the captured launch's work: "<n> scatterings, <n> flight cell visits, <n> peel-off visits"
    m = re.search(r"(\d+) scatterings, (\d+) flight cell visits, (\d+) peel-off visits", text)
    if m:
        s, c, p = (float(v) for v in m.groups())
        out["visits_per_scattering"] = {"cell": c / s, "peel": p / s}
    # the same solves without cameras: the per-scattering work with no peel-off
    try:
        t0 = open(os.path.join(PROFILES, f"k_transport_{name}_nocam.md")).read()
    except OSError:
        t0 = ""
    m0 = re.search(r"kernel_source_sha256: `([0-9a-f]+)`", t0)
    m1 = re.search(r"fp32_flop_per_scattering_no_cameras: ([0-9.eE+-]+)", t0)
    if m0 and m1 and m0.group(1) == kernel_source_hash():
        out["fp32_flop_per_scattering_no_cameras"] = float(m1.group(1))
        out["profile_no_cameras"] = os.path.relpath(os.path.join(PROFILES, f"k_transport_{name}_nocam.md"), ROOT)
    return out


def fp32_peak_tflops(info):
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    return info["sm_count"] * 128 * 2 * sm_max * 1e6 / 1e12, sm_max


def roofline(units, scat, kernel_ms, served_rate, info, launches=1, mix=None):
    """`alu` roofline of the transport kernel: achieved = FP32 operations per
    launch (a per-scattering count x the scatterings of a launch) / the
    launch's average CUDA-event duration, i.e. the FP32 operations of
    `launches` launches over their summed device time; frac_served the same
    count at the served (wall) scattering rate.  The per-scattering count is
    the capture's, for the capture's work mix; with `mix` (flight cell and
    peel-off visits per scattering of the timed region) and a capture of the
    same solves without cameras (F0), it is scaled to the timed region's
    peel-off work: F0 + (F - F0) x (peel visits per scattering here / in the
    capture), the peel-off part of the capture taken per visit."""
    peak, sm_max = fp32_peak_tflops(info)
    src = f"{info['sm_count']} SMs x 128 FP32 lanes x 2 x {sm_max:g} MHz (max SM clock, of measured)"
    if not units or units.get("fp32_flop_per_scattering") is None:
        return {"bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None, "traffic": None,
                "peak_source": src, "note": "no current ncu summary for this kernel"}
    f_capture = units["fp32_flop_per_scattering"]
    f0 = units.get("fp32_flop_per_scattering_no_cameras")
    pv = (units.get("visits_per_scattering") or {}).get("peel")
    model = "the capture's FP32 operations per scattering (its work mix)"
    f = f_capture
    if mix is not None and f0 is not None and pv:
        f = f0 + (f_capture - f0) * mix["peel"] / pv
        model = ("F0 + (F - F0) x peel visits per scattering (timed region / capture): F0 from the capture "
                 "without cameras, F from the capture with them")
    achieved = f * scat / (kernel_ms * 1e-3) / 1e12
    d = units.get("dram_bytes_per_scattering")
    n = max(int(launches), 1)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": d * scat / n if d is not None else None,
            "traffic_unit": "DRAM bytes per launch (the capture's bytes per scattering, at the capture's work mix, "
                            "x a launch's scatterings)",
            "flop_per_scattering": f, "flop_model": model, "flop_per_scattering_capture": f_capture,
            "flop_per_scattering_no_cameras": f0, "frac_served": f * served_rate / 1e12 / peak,
            "launches": {"count": n, "scatterings": scat, "kernel_ms_total": kernel_ms,
                         "kernel_ms_avg": kernel_ms / n},
            "profile": units["profile"], "peak_source": src,
            **({"visits_per_scattering": {"timed_region": mix, "profile": units.get("visits_per_scattering")}}
               if mix is not None else {})}


def served_burst(C, ctx, stream, reqs, read=None, stats=None):
    """Submit every (grid, spec) at once and wait for all: (device ms between
    CUDA events on the library's stream around submit..done, wall s, results
    of colt_read_result (or read(rid, spec)), per-request latency ms).  With
    a dict `stats`, its "longest_history" is set to the most scatterings of
    one packet over all the requests."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    t0 = time.perf_counter()
    ids = list(zip(C.colt_submit_many(ctx, reqs, images=read is not None), [sp for _, sp in reqs]))
    for rid, _ in ids:
        C.colt_wait(ctx, rid, -1.0)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out, lat = [], []
    longest = 0
    for rid, sp in ids:
        st = C.colt_poll(ctx, rid)
        lat.append(st["latency_ms"])
        longest = max(longest, st["longest_history"])
        r = read(rid, sp) if read else C.colt_read_result(ctx, rid, S.RunSpec(**{**sp.__dict__, "cameras": []}))
        out.append(r)
        C.colt_release(ctx, rid)
    if stats is not None:
        stats["longest_history"] = longest
    return ev0.elapsed_time(ev1), wall, out, lat


def pct(xs, q):
    return float(np.percentile(np.asarray(xs, float), q)) if len(xs) else None


def cosmo_specs(srcs, cams, cnb, B, off, cap=None):
    out = []
    for j, (pos, sig) in enumerate(srcs):
        sp = S.RunSpec(n_packets=B, seed=300 + j, src_pos=pos, src_sigma=sig, albedo=0.32, spec_units=1,
                       spec_lo=-1000.0, spec_hi=1000.0, spec_nbins=200, cameras=cams, cam_units=1,
                       cam_lo=-1000.0, cam_hi=1000.0, cam_nbins=cnb, precision=1, pid_offset=off + j * B)
        if cap:
            sp.max_scatter = cap
        out.append(sp)
    return out


def leg_cosmo(C, ctx, stream, args, info, world, rank):
    """Headline: the cosmological box, K steps served together; e2e from the
    same pass (grid from host fields .. results on the host)."""
    import torch
    g, srcs, cams, cnb, label = octree_workload("cosmo")
    B = args.cosmo_packets
    ns = len(srcs)

    def step_specs(s, cap=None):
        return cosmo_specs(srcs, cams, cnb, B, ((s * world + rank) * ns) * B, cap)
    # warm-up on a grid of its own: tuning on capped histories, then W steps
    # with histories capped at 1e4 scatterings
    hw = C.colt_create_grid(ctx, g)
    tuned = C.colt_autotune(ctx, hw, cosmo_specs(srcs[:1], S.axis_cameras(0, ("+x", "+y", "+z")), cnb,
                                                 1 << 16, 1 << 40, cap=2000)[0])
    served_burst(C, ctx, stream, [(hw, sp) for s in range(args.warmup) for sp in step_specs(s, cap=10000)])
    C.colt_destroy_grid(ctx, hw)
    launches0, timed0, kms0, cv0, pv0 = launch_stats(C, ctx, None)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    # the timed pass: e2e region (events e0..e3, with host reads), device region (e1..e2)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    h2d = sum(4 * g.n_cells for _ in range(6)) + g.leaf_level.nbytes + g.leaf_ijk.nbytes
    d2h = 0
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        torch.cuda.synchronize()
        e[0].record(stream)
        h = C.colt_create_grid(ctx, g)
        torch.cuda.synchronize()
        e[1].record(stream)
        reqs = [(h, sp) for s in range(args.warmup, args.warmup + args.steps) for sp in step_specs(s)]
        ids = list(zip(C.colt_submit_many(ctx, reqs), [sp for _, sp in reqs]))
        for rid, _ in ids:
            C.colt_wait(ctx, rid, -1.0)
        e[2].record(stream)
        torch.cuda.synchronize()
        scat = pk = 0
        lat = []
        longest = 0
        for rid, sp in ids:
            st = C.colt_poll(ctx, rid)
            lat.append(st["latency_ms"])
            longest = max(longest, st["longest_history"])
            r = read_with_images(C, ctx, rid, sp)
            d2h += sum(v.nbytes for v in r.values() if isinstance(v, np.ndarray))
            scat += r["n_scat"]
            pk += r["n_emitted"]
            del r
            C.colt_release(ctx, rid)
        C.colt_destroy_grid(ctx, h)
        e[3].record(stream)
        torch.cuda.synchronize()
    launches1, timed1, kms1, cv1, pv1 = launch_stats(C, ctx, None)
    # this rank's work mix in the timed region, beside the captured launch's;
    # the roofline is this rank's launches over their own time
    scat_rank = scat
    mix = {"cell": (cv1 - cv0) / max(scat, 1), "peel": (pv1 - pv0) / max(scat, 1)}
    launches = launches1 - launches0
    ms = e[1].elapsed_time(e[2])
    ms_e2e = e[0].elapsed_time(e[3])
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms, ms_e2e, float(longest)], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_e2e, longest = float(t[0].item()), float(t[1].item()), int(t[2].item())
        c = torch.tensor([scat, pk], device="cuda", dtype=torch.float64)
        dist.all_reduce(c)
        scat, pk = int(c[0].item()), int(c[1].item())
    value = scat / (ms * 1e-3)
    units = profile_units("cosmo")
    return {
        "value": value, "photons_per_s": pk / (ms * 1e-3), "ms": ms, "scat": scat, "packets": pk,
        "longest_history": longest,
        "latency": {"p50": pct(lat, 50), "p99": pct(lat, 99), "n_requests": len(lat),
                    "arrivals": "burst: the K steps' solves submitted together"},
        "e2e": {"value": scat / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d // args.steps),
                "d2h_bytes_per_step": int(d2h // args.steps), "ms_per_step": ms_e2e / args.steps,
                "steps": args.steps,
                "path": "colt_create_grid from host fields (once, bytes spread over the steps) -> colt_submit_many "
                        "of every step -> colt_wait -> colt_read_result with escape spectra, camera spectra and "
                        "image cubes -> colt_destroy_grid"},
        "roofline": roofline(units, scat_rank, kms1 - kms0, value / max(world, 1), info, launches=timed1 - timed0,
                             mix=mix),
        "gpu_launches": launches, "clocks": clk.summary(),
        "config": {"workload": label, "sources": ns, "packets_per_source_per_step": B,
                   "cameras": "3 x 512^2 x 256 (+x, +y, +z)",
                   "grid": f"octree, {g.n_cells} leaves, levels {int(g.leaf_level.min())}-{int(g.leaf_level.max())} "
                           f"(refined on density; the workload description names levels 7-14, the density "
                           f"criterion of this generator stops at 12)",
                   "precision": "mixed (FP32 transport, FP32-pair position and tau, FP64 escape and tallies)",
                   "launch": "served: the K steps submitted together (colt_submit_many), persistent launches in flight",
                   "launch_config": dict(tuned, source="colt_autotune on one source, 65536 packets capped at "
                                                       "2000 scatterings"),
                   "warmup": "W steps with histories capped at 1e4 scatterings",
                   "l2": "records 300 MB + octree tables 265 MB + tallies 1.6 GB per solve > 129 MB L2: "
                         "inputs larger than L2"},
    }


def leg_sphere(C, ctx, stream, args, info):
    """The 128^3 sphere suite: served steps, the plain launch of the whole
    job, the plain FP64 kernel on one solve."""
    grids = [case_grid(t, v) for t, v in cases()]
    hs = [C.colt_create_grid(ctx, g) for g in grids]
    B = 125000
    tuned = C.colt_autotune(ctx, hs[4], case_spec(4, B, 0, images=False))

    def specs_of(s):
        return [case_spec(i, B, s * B, images=True) for i in range(9)]
    served_burst(C, ctx, stream, [(hs[i], sp) for i, sp in enumerate(specs_of(0))])
    with ClockSampler(0) as clk:
        ms, wall, res, lat = served_burst(C, ctx, stream, [(hs[i], sp) for s in range(1, 1 + args.sphere_steps)
                                                           for i, sp in enumerate(specs_of(s))])
        scat = sum(r["n_scat"] for r in res)
        pk = sum(r["n_emitted"] for r in res)
        # plain: the whole job (1e6 packets per case) in one launch
        job = [case_spec(i, PACKETS_PER_CASE_JOB, 10 ** 8, images=True) for i in range(9)]
        plain = C.colt_run_batch(ctx, hs, job, images=True, outputs=False)
        # plain FP64: one solve (tau0 = 1e5, static) alone
        sp64 = case_spec(1, args.fp64_packets, 2 * 10 ** 8, images=True)
        sp64.precision = 0
        p64 = C.colt_run(ctx, hs[1], sp64)
    for h in hs:
        C.colt_destroy_grid(ctx, h)
    plain_scat = sum(r["n_scat"] for r in plain)
    plain_ms = plain[0]["kernel_ms"]
    value = scat / (ms * 1e-3)
    units = profile_units("sphere128")
    return {"value": value, "unit": UNIT, "photons_per_s": pk / (ms * 1e-3), "steps": args.sphere_steps,
            "ms_per_step": ms / args.sphere_steps,
            "served_latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "n_requests": len(lat),
                                  "arrivals": "burst"},
            "plain": {"value": plain_scat / (plain_ms * 1e-3), "unit": UNIT, "kernel_ms": plain_ms,
                      "scatterings": plain_scat, "packets": 9 * PACKETS_PER_CASE_JOB,
                      "path": "colt_run_batch: the whole job (1e6 packets per case, nine cases) in one launch",
                      "cell_visits": plain[0]["n_cell_visits"], "peel_visits": plain[0]["n_peel_visits"]},
            "plain_fp64": {"value": p64["n_scat"] / (p64["kernel_ms"] * 1e-3), "unit": UNIT,
                           "kernel_ms": p64["kernel_ms"], "packets": args.fp64_packets,
                           "path": "colt_run, precision PLAIN: one solve (tau0 = 1e5, static) per launch"},
            "roofline": roofline(units, plain_scat, plain_ms, value, info,
                                 mix={"cell": plain[0]["n_cell_visits"] / max(plain_scat, 1),
                                      "peel": plain[0]["n_peel_visits"] / max(plain_scat, 1)}),
            "clocks": clk.summary(),
            "config": {"workload": WORKLOAD, "packets_per_case_per_step": B,
                       "cameras": "6 x 128^2 x 200", "precision": "mixed (served, plain); FP64 (plain_fp64)",
                       "launch_config": dict(tuned, source="colt_autotune on the tau0=1e6 static case"),
                       "l2": "records 9 x 67 MB + tallies 9 x 157 MB per step > 129 MB L2"}}


def leg_halo(C, ctx, stream, args, info):
    g, srcs, cams, cnb, label = octree_workload("halo")
    pos, sig = srcs[0]
    h = C.colt_create_grid(ctx, g)
    B = args.halo_packets

    def spec(s, cap=None):
        sp = S.RunSpec(n_packets=B, seed=300, src_pos=pos, src_sigma=sig, albedo=0.32, spec_units=1,
                       spec_lo=-1000.0, spec_hi=1000.0, spec_nbins=200, cameras=cams, cam_units=1,
                       cam_lo=-1000.0, cam_hi=1000.0, cam_nbins=cnb, precision=1, pid_offset=s * B)
        if cap:
            sp.max_scatter = cap
        return sp
    served_burst(C, ctx, stream, [(h, spec(0, cap=10000))])
    tail = {}
    with ClockSampler(0) as clk:
        ms, wall, res, lat = served_burst(C, ctx, stream, [(h, spec(s)) for s in range(1, 1 + args.halo_steps)],
                                          stats=tail)
    C.colt_destroy_grid(ctx, h)
    scat = sum(r["n_scat"] for r in res)
    pk = sum(r["n_emitted"] for r in res)
    return {"value": scat / (ms * 1e-3), "unit": UNIT, "photons_per_s": pk / (ms * 1e-3), "steps": args.halo_steps,
            "ms_per_step": ms / args.halo_steps, "longest_history_scatterings": tail["longest_history"],
            "served_latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "n_requests": len(lat),
                                  "arrivals": "burst"},
            "clocks": clk.summary(),
            "config": {"workload": label, "packets_per_step": B, "cameras": "6 x 128^2 x 200",
                       "grid": f"octree, {g.n_cells} leaves, levels {int(g.leaf_level.min())}-"
                               f"{int(g.leaf_level.max())}", "precision": "mixed",
                       "launch": "served: the steps submitted together"}}


def leg_serving(C, ctx, stream, args, n_req=256, load=0.75):
    reqs = serving_requests(n_req)
    grids = [C.colt_create_grid(ctx, serving_grid(q)) for q in reqs]
    specs = [S.RunSpec(n_packets=q["n"], seed=q["seed"], albedo=0.32, spec_units=1, spec_lo=-q["w"],
                       spec_hi=q["w"], spec_nbins=200, precision=1) for q in reqs]
    t0 = time.perf_counter()
    cal = served_burst(C, ctx, stream, list(zip(grids, specs)), read=lambda rid, sp: C.colt_read_result(ctx, rid, sp))
    t_batch = time.perf_counter() - t0
    rate = load * n_req / cal[1]
    arr = np.cumsum(np.random.default_rng(4).exponential(1.0 / rate, n_req))
    import torch
    with ClockSampler(0) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        t0 = time.perf_counter()
        rids = []
        for i in range(n_req):
            while time.perf_counter() - t0 < arr[i]:
                if rids:
                    C.colt_poll(ctx, rids[-1])          # drive the scheduler between arrivals
                time.sleep(0.0005)
            rids.append(C.colt_submit(ctx, grids[i], specs[i]))
        done = []
        for rid, sp in zip(rids, specs):
            C.colt_wait(ctx, rid, -1.0)
        ev1.record(stream)
        torch.cuda.synchronize()
    for rid, sp in zip(rids, specs):
        done.append((C.colt_poll(ctx, rid), C.colt_read_result(ctx, rid, sp)))
        C.colt_release(ctx, rid)
    ms = ev0.elapsed_time(ev1)
    scat = sum(r["n_scat"] for _, r in done)
    lat = [st["latency_ms"] for st, _ in done]
    same = all(np.array_equal(a["spec"], b["spec"]) for a, (_, b) in zip(cal[2], done))
    # the requests slowest in the mix, each solved alone (blocking launch): a
    # lower bound of the longest single request's own time
    slow = sorted(range(n_req), key=lambda i: -lat[i])[:5]
    alone = {}
    for i in slow:
        r = C.colt_run(ctx, grids[i], specs[i])
        alone[i] = r["kernel_ms"]
    out = {"value": scat / (ms * 1e-3), "unit": UNIT,
           "photons_per_s": sum(r["n_emitted"] for _, r in done) / (ms * 1e-3),
           "served_latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": float(max(lat)),
                                 "n_requests": n_req,
                                  "arrivals": f"Poisson, {rate:.3f} requests/s = {load:.2f} x the all-at-once "
                                              f"throughput ({n_req} requests in {cal[1]:.1f} s)"},
            "slowest_alone_ms": {str(i): alone[i] for i in slow},
            "longest_alone_ms": float(max(alone.values())),
            "batch_all_at_once": {"wall_s": cal[1], "latency_ms": {"p50": pct(cal[3], 50), "p99": pct(cal[3], 99)}},
            "results_identical_across_mixes": same, "clocks": clk.summary(),
            "config": {"workload": f"serving_mix_{n_req}req_64cubed", "precision": "mixed",
                       "admission": "memory budget (90% of free HBM)"}}
    for h in grids:
        C.colt_destroy_grid(ctx, h)
    return out


def oracle_sample_cosmo(target_s=15.0, cores=0):
    """The FP64 oracle, as it stands, on a bounded sample of the headline
    workload: packets of the five sources (camera spectra, no images), the
    grid derived once; the packet loop timed."""
    import oracle as O
    g, srcs, cams, cnb, label = octree_workload("cosmo")
    cams0 = [S.Camera(c.direction, 0) for c in cams]
    n = 2
    while True:
        specs = cosmo_specs(srcs, cams0, cnb, n, 10 ** 9)
        t0 = time.perf_counter()
        rs = O.run_many(g, specs, workers=5)
        t = time.perf_counter() - t0
        if t > target_s / 3 or n >= 1 << 12:
            break
        n *= 2
    scat = sum(r["n_scat"] for r in rs)
    return dict(value=scat / t, unit=UNIT, cores=os.cpu_count(), photons_per_s=5 * n / t, seconds=t, kind="oracle",
                sample=f"{5 * n} packets ({n} per source) of {label}, three cameras' spectra (no images), five "
                       f"sources run side by side on the host cores; the packet loop timed, grid derivation excluded "
                       f"as on the GPU")


def run_suite(args):
    import torch
    from paper_1409_4480_gb300 import colt as C
    world, rank, local = _rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = C.colt_init(local, 0, stream.cuda_stream)
    info = C.colt_device_info(ctx)
    head = leg_cosmo(C, ctx, stream, args, info, world, rank)
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "photons_per_s": head["photons_per_s"], "served_latency_ms": head["latency"], "config": head["config"],
            "gpu_launches": head["gpu_launches"], "roofline": head["roofline"], "e2e": head["e2e"],
            "clocks": head["clocks"],
            "counts": {"scatterings": head["scat"], "packets": head["packets"],
                       "longest_history_scatterings": head["longest_history"]}}
    if rank == 0 and world == 1:
        wl = {}
        if not args.no_secondary:
            wl["sphere128"] = leg_sphere(C, ctx, stream, args, info)
            wl["halo"] = leg_halo(C, ctx, stream, args, info)
            wl["serving"] = leg_serving(C, ctx, stream, args)
        line["workloads"] = wl
        if not args.no_cpu:
            line["cpu_baseline"] = oracle_sample_cosmo(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    C.colt_finalize(ctx)
    if dist:
        dist.destroy_process_group()




def run_profile_case(args):
    """One short launch of a workload with histories capped (ncu capture
    driver): prints the launch's counters as JSON."""
    from paper_1409_4480_gb300 import colt as C
    ctx = C.colt_init(0)
    name = args.profile_case
    if name == "sphere128":
        hs = [C.colt_create_grid(ctx, case_grid(t, v)) for t, v in cases()]
        specs = [case_spec(i, 16384, 0, images=True) for i in range(9)]
    else:
        g, srcs, cams, cnb, label = octree_workload(name)
        h = C.colt_create_grid(ctx, g)
        if name == "cosmo":
            # one source (a few GB on the device: the grid and one solve's image cubes)
            specs = cosmo_specs(srcs[:1], cams, cnb, 65536, 0)
        else:
            pos, sig = srcs[0]
            specs = [S.RunSpec(n_packets=65536, seed=300, src_pos=pos, src_sigma=sig, albedo=0.32, spec_units=1,
                               spec_lo=-1000.0, spec_hi=1000.0, spec_nbins=200, cameras=cams, cam_units=1,
                               cam_lo=-1000.0, cam_hi=1000.0, cam_nbins=cnb, precision=1)]
        hs = [h] * len(specs)
    for sp in specs:
        sp.max_scatter = 2000
        if args.profile_no_cameras:
            sp.cameras = []     # the same histories (peel-off draws no random numbers), no peel-off work
    r = C.colt_run_batch(ctx, hs, specs, images=True, outputs=False)
    print(json.dumps({"workload": name, "launches": 1, "kernel_ms": r[0]["kernel_ms"],
                      "scatterings": sum(x["n_scat"] for x in r), "packets": sum(x["n_emitted"] for x in r),
                      "cell_visits": r[0]["n_cell_visits"], "peel_visits": r[0]["n_peel_visits"],
                      "peel_rays": r[0]["n_peel_rays"], "max_scatter": 2000,
                      "cameras": 0 if args.profile_no_cameras else len(specs[0].cameras),
                      "kernel_source_sha256": kernel_source_hash()}), flush=True)
    C.colt_finalize(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="colt", choices=["colt", "reference"])
    ap.add_argument("--workload", default="suite",
                    choices=["suite", "sphere128", "halo", "halo_diffuse", "cosmo", "serving", "tslab", "galaxies"])
    ap.add_argument("--core-skip", type=int, default=1, choices=[0, 1, 2],
                    help="octree and galaxy workloads: a tau_0 for x_crit (1 cell + non-local, 2 Jeans)")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--load", type=float, default=0.75)
    ap.add_argument("--packets-per-case", type=int, default=None,
                    help="single-workload modes: packets per solve per step (default: 125000 for the sphere suite "
                         "and --single-case; 4096 halo / halo_diffuse / galaxies, 2048 cosmo, 20000 tslab)")
    ap.add_argument("--cosmo-packets", type=int, default=1024, help="suite headline: packets per source per step")
    ap.add_argument("--halo-packets", type=int, default=8192, help="suite: halo packets per step")
    ap.add_argument("--halo-steps", type=int, default=8, help="suite: halo steps")
    ap.add_argument("--sphere-steps", type=int, default=6, help="suite: sphere-suite steps")
    ap.add_argument("--fp64-packets", type=int, default=100000, help="suite: packets of the plain FP64 solve")
    ap.add_argument("--no-secondary", action="store_true", help="suite: the headline alone")
    ap.add_argument("--ref-packets", type=int, default=16)
    ap.add_argument("--single-case", type=int, default=-1)
    ap.add_argument("--profile-case", default=None, choices=["cosmo", "sphere128", "halo"])
    ap.add_argument("--profile-no-cameras", action="store_true",
                    help="with --profile-case: the same solves without cameras (no peel-off work)")
    ap.add_argument("--max-scatter", type=int, default=0)
    ap.add_argument("--no-images", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.packets_per_case is None:
        args.packets_per_case = {"halo": 4096, "halo_diffuse": 4096, "galaxies": 4096, "cosmo": 2048,
                                 "tslab": 20000}.get(args.workload, 125000)
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.single_case >= 0:
        run_single_case(args)
    elif args.workload == "suite":
        run_suite(args)
    elif args.workload in ("halo", "halo_diffuse", "cosmo"):
        run_octree(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "tslab":
        run_slab_suite(args)
    elif args.workload == "galaxies":
        run_galaxies(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
