"""Benchmark of the Lyman-alpha packet transport on one (or N) GB300.

Workload (the 128^3 expanding/contracting dusty sphere suite): a uniform
128^3 sphere at T = 1e4 K, tau0 in {1e5, 1e6, 1e7}, Hubble-like velocity with
v_max in {-200, 0, +200} km/s (nine cases), dust tau_d = 1 with albedo 0.32,
peel-off to six axis cameras of 128^2 pixels x 200 bins over +-1000 km/s,
1e6 packets per case for the whole job.  A step is one batch of packets of
all nine cases in one persistent launch (colt_run_batch, mixed precision);
the job is steps_per_job batches.  Inputs are synthetic (seeded generators).

value      scatterings/s (executed, core-skipped ones not counted), whole job
e2e        the same metric through colt_solve with host fields: grid upload +
           records + non-local a*tau + transport + result download per step
--impl reference   the FP64 CPU oracle on the host cores, bounded samples
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
    O.run(g, case_spec(i, 4, 0, images=False), n_threads=cores)  # build + warm
    while True:
        r = O.run(g, case_spec(i, n, 0, images=False), n_threads=cores)
        if r["seconds"] > target_s / 4 or n >= 1 << 20:
            break
        n *= 4
    if r["seconds"] < target_s:
        n = int(n * target_s / max(r["seconds"], 1e-3))
        r = O.run(g, case_spec(i, n, 0, images=False), n_threads=cores)
    return dict(value=r["n_scat"] / r["seconds"], unit=UNIT, cores=r["n_threads"],
                photons_per_s=n / r["seconds"], seconds=r["seconds"],
                sample=f"{n} packets of the tau0={case[0]:g}, v_max={case[1]:g} km/s case (6 cameras x 200 "
                       f"bins peel-off, no images), one oracle call incl. grid derivation and a*tau_NL")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    steps_rates = []
    cores = os.cpu_count()
    t_all = 0.0
    n_scat = 0
    n_pk = 0
    for s in range(args.warmup + args.steps):
        t, v = cases()[s % 9]
        g = case_grid(t, v)
        spec = case_spec(s % 9, args.ref_packets, s * args.ref_packets, images=False)
        r = O.run(g, spec)
        if s >= args.warmup:
            t_all += r["seconds"]
            n_scat += r["n_scat"]
            n_pk += args.ref_packets
            steps_rates.append(r["n_scat"] / r["seconds"])
    value = n_scat / t_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "photons_per_s": n_pk / t_all,
            "config": {"workload": "sphere128_T1e4_dust1_9cases_6cam", "cases": "tau0 {1e5,1e6,1e7} x v_max {-200,0,200}",
                       "packets_per_step": args.ref_packets, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_packets} packets per step, one case per step cycling through the 9"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg --
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
    # grids resident in HBM before the timed region
    grids_h = [case_grid(t, v) for t, v in cases()]
    hs = [C.colt_create_grid(ctx, g) for g in grids_h]
    img = not args.no_images

    def step(s):
        # packet ids of this (step, rank): weak scaling, disjoint ranges
        off = (s * world + rank) * B
        specs = [case_spec(i, B, off, images=img) for i in range(9)]
        return C.colt_run_batch(ctx, hs, specs, images=img, outputs=False)

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot_scat = tot_pk = 0
    kms = []
    visits = [0, 0, 0]
    with ClockSampler(local) as clk:
        ev0.record(stream)
        t0 = time.perf_counter()
        for s in range(args.warmup, args.warmup + args.steps):
            res = step(s)
            tot_scat += sum(r["n_scat"] for r in res)
            tot_pk += sum(r["n_emitted"] for r in res)
            kms.append(res[0]["kernel_ms"])
            visits[0] += res[0]["n_cell_visits"]
            visits[1] += res[0]["n_peel_visits"]
            visits[2] += res[0]["n_peel_rays"]
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        c = torch.tensor([tot_scat, tot_pk], device="cuda", dtype=torch.float64)
        dist.all_reduce(c)
        tot_scat, tot_pk = int(c[0].item()), int(c[1].item())
    value = tot_scat / (ms / 1e3)
    photons = tot_pk / (ms / 1e3)

    # end to end: host fields, colt_solve per case (upload, records, a*tau_NL,
    # transport, download of spectra and image cubes), one step
    e2e = None
    if not args.no_e2e:
        h2d = d2h = 0
        t0 = time.perf_counter()
        e2e_scat = 0
        ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev2.record(stream)
        s = args.warmup + args.steps
        for i, g in enumerate(grids_h):
            sp = case_spec(i, B, (s * world + rank) * B, images=img)
            r = C.colt_solve(ctx, g, sp, images=img)
            e2e_scat += r["n_scat"]
            h2d += 6 * 4 * g.n_cells
            d2h += r["spec"].nbytes + r["cam_spec"].nbytes + r["cam_spec2"].nbytes + (r["cam_image"].nbytes if img else 0)
        ev3.record(stream)
        torch.cuda.synchronize()
        e2e_ms = ev2.elapsed_time(ev3)
        e2e = {"value": e2e_scat / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
               "path": "colt_solve (host fields -> device records -> a*tau_NL -> transport -> host results)"}

    # roofline of the transport kernel: FP32 issue-bound
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = info["sm_count"] * 128 * 2 * sm_max * 1e6 / 1e12
    kern_ms = statistics.mean(kms)
    ops = (args.flops_peel * visits[1] + args.flops_cell * visits[0] + args.flops_scat * tot_scat / world) / args.steps
    achieved = ops / (kern_ms / 1e3) / 1e12
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(args.cpu_seconds)
        cpu["kind"] = "oracle"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "photons_per_s": photons,
            "config": {"workload": "sphere128_T1e4_dust1_9cases_6cam",
                       "cases": "tau0 {1e5,1e6,1e7} x v_max {-200,0,200} km/s, tau_d=1, A=0.32",
                       "packets_per_case_per_step": B, "steps_per_job": PACKETS_PER_CASE_JOB // B,
                       "cameras": "6 x 128^2 x 200" if img else "6 x 200 (no images)",
                       "grid": "128^3 Cartesian, 32 B records", "precision": "mixed (FP32 transport, FP64 tau/escape)",
                       "launch": "colt_run_batch: one persistent launch of all 9 cases per step",
                       "l2": "records 9 x 67 MB + tallies 9 x 157 MB > 129 MB L2: inputs larger than L2"},
            "gpu_launches": args.steps,
            "kernel_ms_mean": kern_ms,
            "counts": {"scatterings": tot_scat, "packets": tot_pk, "cell_visits": visits[0],
                       "peel_visits": visits[1], "peel_rays": visits[2]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": None,
                         "peak_source": f"{info['sm_count']} SMs x 128 FP32 lanes x 2 x {sm_max:g} MHz (max SM clock of measured)"},
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="colt", choices=["colt", "reference"])
    ap.add_argument("--packets-per-case", type=int, default=1 << 15)
    ap.add_argument("--ref-packets", type=int, default=64)
    ap.add_argument("--no-images", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    # algorithmic FP32 operations per unit (the design doc derives them from the code)
    ap.add_argument("--flops-peel", type=float, default=30.0)
    ap.add_argument("--flops-cell", type=float, default=45.0)
    ap.add_argument("--flops-scat", type=float, default=300.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
