"""Full-history statistical parity with the FP64 oracle on the five workloads
at their own sizes (grids, cameras and image resolutions of the benchmark).

Transport is chaotic, so complete histories are compared as samples: the CUDA
path (mixed precision, as benchmarked; FP64 as well for the 32^3 sphere) and
the oracle run disjoint packet-id ranges.  For every solve:
  * escape fraction: two-sample binomial, |z| <= 3;
  * escape spectrum: two-sample chi-square of the counts (sparse bins merged);
  * camera spectra and images: both sides run as batches of the same number
    of packets, so that under the null hypothesis the batches are
    exchangeable; a permutation test over the batches compares the
    per-packet bin means (peel-off weights are heavy-tailed and the
    contributions of one packet correlated, which rules out normal
    approximations).  Spectral bins are merged to >= 30 effective
    contributions a side; images are compared in pixel blocks: both sides
    tally at the block resolution, and separately the full-resolution GPU
    image of the same packets, pooled into those blocks, must equal the GPU's
    block-resolution image (camera resolution does not touch the histories),
    which carries the full-resolution image path to the oracle.
Every p-value must exceed 0.01/m, m the number of p-values of the workload
(family-wise level 1%, Bonferroni).  The oracle of a workload runs in a
thread of its own, overlapping the GPU side (the C oracle releases the GIL).
Each test prints one `PARITY {...}` line with the measured differences.

Sec. 3.1-3.2 (the method), Sec. 6.1, Eq. SB (peel-off), Sec. 4.1-4.2 (the
test problems these workloads generalise).
"""
import json
import threading

import numpy as np
import pytest

import parity_stats as PS
from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(colt):
    c = colt.colt_init(0)
    yield c
    colt.colt_finalize(c)


class OracleThread:
    """Oracle runs in a background thread: groups of (grid, [specs], images),
    each group on one grid derivation (O.run_many); results in order."""

    def __init__(self, O, groups, workers=4):
        self.groups, self.res, self.err = groups, [], []
        self.th = threading.Thread(target=self._work, args=(O, workers), daemon=True)
        self.th.start()

    def _work(self, O, workers):
        try:
            for g, specs, im in self.groups:
                self.res += O.run_many(g, specs, images=im, workers=workers)
        except BaseException as e:   # noqa: BLE001 -- re-raised in join()
            self.err.append(e)

    def join(self):
        self.th.join()
        if self.err:
            raise self.err[0]
        return self.res


def gpu_served(colt, ctx, reqs, block_pix=None):
    """Submit every (grid handle, spec) at once to the serving scheduler; read
    counters and spectra, and with block_pix the image cubes pooled into
    block_pix-pixel blocks per camera."""
    ids = [colt.colt_submit(ctx, h, sp, images=block_pix is not None) for h, sp in reqs]
    for rid in ids:
        colt.colt_wait(ctx, rid, -1.0)
    out = []
    for rid, (h, sp) in zip(ids, reqs):
        r = colt.colt_read_result(ctx, rid, sp)
        if block_pix is not None:
            r["blocks"] = np.concatenate([
                PS.block_image(colt.colt_read_image(ctx, rid, c, cam.npix, sp.cam_nbins), cam.npix, sp.cam_nbins,
                               block_pix) for c, cam in enumerate(sp.cameras)])
        colt.colt_release(ctx, rid)
        out.append(r)
    return out


def pooling_check(colt, ctx, h, pairs, block_pix):
    """The same packets with full-resolution and block-resolution cameras
    (pairs of specs, all submitted together): identical histories (integer
    tallies equal), and the full-resolution image pooled into blocks equals
    the block-resolution image up to events on a block edge (pixel
    coordinates are FP32).  Returns the relative L1 difference per pair."""
    full = gpu_served(colt, ctx, [(h, f) for f, _ in pairs], block_pix=block_pix)
    blk = gpu_served(colt, ctx, [(h, b) for _, b in pairs], block_pix=1)
    out = []
    for a, b in zip(full, blk):
        assert np.array_equal(a["spec"], b["spec"]) and a["n_scat"] == b["n_scat"]
        assert np.allclose(a["cam_spec"], b["cam_spec"], rtol=1e-9, atol=1e-300)
        d = float(np.abs(a["blocks"] - b["blocks"]).sum() / max(b["blocks"].sum(), 1e-300))
        assert d <= 1e-4, d
        out.append(d)
    return out


def oracle_blocks(r, spec, nblk):
    """The oracle's image tallied at nblk x nblk pixels per camera, flattened."""
    return np.asarray(r["cam_image"]).reshape(len(spec.cameras), nblk, nblk, spec.cam_nbins).sum(axis=3).ravel()


def add_results(rs):
    """Tallies of several solves of one batch (sources of one step) added."""
    out = {k: sum(r[k] for r in rs) for k in ("n_emitted", "n_escaped", "n_absorbed", "n_capped", "n_scat")}
    out["spec"] = np.sum([r["spec"] for r in rs], axis=0)
    for k in ("cam_spec", "cam_spec2", "blocks"):
        if k in rs[0]:
            out[k] = np.sum([r[k] for r in rs], axis=0)
    return out


def compare(label, gb, ob, cams=True, images=False, alpha=0.01):
    """Statistical comparison of GPU batches gb with oracle batches ob (lists
    of result dicts, blocks already pooled).  Returns the report and the list
    of p-values; asserts the binomial and family-wise chi-square criteria."""
    rep = {"workload": label, "gpu_packets": int(sum(r["n_emitted"] for r in gb)),
           "oracle_packets": int(sum(r["n_emitted"] for r in ob)), "batches": [len(gb), len(ob)]}
    ng, no = rep["gpu_packets"], rep["oracle_packets"]
    kg, ko = sum(r["n_escaped"] for r in gb), sum(r["n_escaped"] for r in ob)
    z, se = PS.binomial_sigma(kg, ng, ko, no)
    rep.update(f_esc_gpu=kg / ng, f_esc_oracle=ko / no, f_esc_z=float(z))
    rep["scat_per_packet"] = [sum(r["n_scat"] for r in gb) / ng, sum(r["n_scat"] for r in ob) / no]
    pv = []
    chi2, dof, p = PS.two_sample_counts(np.sum([r["spec"] for r in gb], axis=0),
                                        np.sum([r["spec"] for r in ob], axis=0))
    rep["spec"] = dict(chi2=chi2, dof=dof, p=p)
    pv.append(p)
    if cams:
        cr = PS.camera_permutation_test([(r["cam_spec"], r["cam_spec2"], r["n_emitted"]) for r in gb],
                                        [(r["cam_spec"], r["cam_spec2"], r["n_emitted"]) for r in ob])
        rep["cameras"] = cr
        pv += [c["p"] for c in cr]
    if images:
        xg = np.array([r["blocks"] / r["n_emitted"] for r in gb])
        xo = np.array([r["blocks"] / r["n_emitted"] for r in ob])
        nblk, T, p = PS.permutation_test(xg, xo)
        mg, mo = xg.mean(axis=0), xo.mean(axis=0)
        rep["image_blocks"] = dict(blocks=nblk, T=T, p=p,
                                   rel_l1=float(np.abs(mg - mo).sum() / max(np.abs(mo).sum(), 1e-300)))
        pv.append(p)
    rep["min_p"] = float(min(pv))
    return rep, pv


def check(reports, pvals, alpha=0.01):
    print("PARITY " + json.dumps(reports, default=float))
    m = len(pvals)
    for rep in reports:
        assert abs(rep["f_esc_z"]) <= 3.0, rep
    assert min(pvals) > alpha / m, (min(pvals), m)


# ------------------------------------------------------------- workloads --
def test_cfg1_sphere32_full_histories(O, colt, ctx):
    """32^3 static sphere, T = 10 K, tau0 = 1e5, 1e3 packets a batch, FP64 (the
    workload's precision) and mixed precision, 100 bins over x in [-40, 40]."""
    g = S.sphere(32, 10.0, 1e5)

    def spec(seed, off, n, prec):
        return S.RunSpec(n_packets=n, seed=seed, T_ref=10.0, spec_units=0, spec_lo=-40, spec_hi=40, spec_nbins=100,
                         precision=prec, pid_offset=off)
    Bg, Bo, n = 12, 8, 1000
    ot = OracleThread(O, [(g, [spec(1, 10 ** 6 + b * n, n, 0) for b in range(Bo)], False)])
    h = colt.colt_create_grid(ctx, g)
    reps, pv = [], []
    try:
        gpu = {prec: gpu_served(colt, ctx, [(h, spec(1, b * n, n, prec)) for b in range(Bg)]) for prec in (0, 1)}
    finally:
        colt.colt_destroy_grid(ctx, h)
    ob = ot.join()
    for prec in (0, 1):
        rep, p = compare(f"sphere32_T10_tau1e5_{'fp64' if prec == 0 else 'mixed'}", gpu[prec], ob, cams=False)
        assert rep["f_esc_gpu"] == 1.0 and rep["f_esc_oracle"] == 1.0     # no dust: every packet escapes
        reps.append(rep)
        pv += p
    check(reps, pv)


def test_cfg2_sphere128_nine_cases(O, colt, ctx):
    """The 128^3 dusty-sphere suite: tau0 {1e5, 1e6, 1e7} x v_max {-200, 0, 200}
    km/s, dust tau 1 with A = 0.32, six cameras of 128^2 pixels x 200 bins.
    Per case: GPU 48 batches and oracle 8 batches of 200 packets, cameras at
    16^2 blocks of 8^2 pixels; the 128^2 images of 4096 GPU packets pooled
    against their 16^2 tally."""
    import bench
    Bg, Bo, n, blk = 48, 8, 200, 8
    nb = 128 // blk
    grids = [bench.case_grid(t, v) for t, v in bench.cases()]

    def spec(i, off, m, npix):
        sp = bench.case_spec(i, m, off, images=True)
        sp.cameras = S.axis_cameras(npix)
        return sp
    ot = OracleThread(O, [(grids[i], [spec(i, 10 ** 7 + b * n, n, nb) for b in range(Bo)], True) for i in range(9)])
    hs = [colt.colt_create_grid(ctx, g) for g in grids]
    pooled = []
    try:
        res = gpu_served(colt, ctx, [(hs[i], spec(i, b * n, n, nb)) for i in range(9) for b in range(Bg)],
                         block_pix=1)
        for i in (4, 8):
            pooled += pooling_check(colt, ctx, hs[i], [(spec(i, 5 * 10 ** 6, 4096, 128),
                                                        spec(i, 5 * 10 ** 6, 4096, nb))], blk)
    finally:
        for h in hs:
            colt.colt_destroy_grid(ctx, h)
    ores = ot.join()
    reps, pv = [], []
    for i, (t, v) in enumerate(bench.cases()):
        gb = res[i * Bg:(i + 1) * Bg]
        ob = ores[i * Bo:(i + 1) * Bo]
        for r in ob:
            r["blocks"] = oracle_blocks(r, spec(i, 0, n, nb), nb)
        rep, p = compare(f"sphere128_tau{t:g}_v{v:g}", gb, ob, cams=True, images=True)
        reps.append(rep)
        pv += p
    reps[0]["pooling_rel_l1"] = pooled
    check(reps, pv)


def test_cfg3_octree_halo(O, colt, ctx):
    """The synthetic AMR halo (2.05e6 leaves, levels 6-12), central Gaussian
    source of 0.1 kpc, six cameras of 128^2 x 200: GPU 48 batches and oracle
    8 batches of 40 packets (about 9e5 scatterings a packet), cameras at 16^2
    blocks; the 128^2 images of 512 GPU packets pooled against their 16^2
    tally."""
    import bench
    g, srcs, cams, cnb, label = bench.octree_workload("halo")
    pos, sig = srcs[0]
    Bg, Bo, n, blk = 48, 8, 40, 8
    nb = 128 // blk

    def spec(off, m, npix):
        return S.RunSpec(n_packets=m, seed=300, src_pos=pos, src_sigma=sig, albedo=0.32, spec_units=1,
                         spec_lo=-1000.0, spec_hi=1000.0, spec_nbins=200, cameras=S.axis_cameras(npix), cam_units=1,
                         cam_lo=-1000.0, cam_hi=1000.0, cam_nbins=cnb, precision=1, pid_offset=off)
    ot = OracleThread(O, [(g, [spec(10 ** 7 + b * n, n, nb) for b in range(Bo)], True)], workers=8)
    h = colt.colt_create_grid(ctx, g)
    try:
        gb = gpu_served(colt, ctx, [(h, spec(b * n, n, nb)) for b in range(Bg)], block_pix=1)
        pooled = pooling_check(colt, ctx, h, [(spec(5 * 10 ** 6, 512, 128), spec(5 * 10 ** 6, 512, nb))], blk)
    finally:
        colt.colt_destroy_grid(ctx, h)
    ob = ot.join()
    for r in ob:
        r["blocks"] = oracle_blocks(r, spec(0, n, nb), nb)
    rep, pv = compare(label, gb, ob, cams=True, images=True)
    rep["pooling_rel_l1"] = pooled
    assert rep["f_esc_gpu"] == 1.0 and rep["f_esc_oracle"] == 1.0        # no dust
    check([rep], pv)


def test_cfg4_serving_mix_sample(O, colt, ctx):
    """A sample of the 256-request serving mix (spheres and slabs on 64^3,
    tau0 1e4-1e8, T 10-1e5 K, v_max +-300 km/s, dust tau 0-2): the first 32
    requests run served together with their own parameters (packet counts
    capped at 1e5); eight of them, spread over the mix, against the oracle
    (6 batches of 100 packets)."""
    import bench
    reqs = bench.serving_requests(32)
    grids = [bench.serving_grid(q) for q in reqs]
    check_ids = [i for i in range(32) if reqs[i]["tau0"] <= 3e7][:8]
    Bo, no, Bg = 6, 100, 4

    def spec(q, n, off):
        return S.RunSpec(n_packets=n, seed=q["seed"], albedo=0.32, spec_units=1, spec_lo=-q["w"], spec_hi=q["w"],
                         spec_nbins=200, precision=1, pid_offset=off)
    ot = OracleThread(O, [(grids[i], [spec(reqs[i], no, 10 ** 7 + b * no) for b in range(Bo)], False)
                          for i in check_ids])
    hs = [colt.colt_create_grid(ctx, gr) for gr in grids]
    try:
        sub = []
        for i, q in enumerate(reqs):
            n = min(q["n"], 100000)
            per = n // Bg if i in check_ids else n
            sub += [(hs[i], spec(q, per, b * per)) for b in range(Bg if i in check_ids else 1)]
        res = gpu_served(colt, ctx, sub)
    finally:
        for h in hs:
            colt.colt_destroy_grid(ctx, h)
    ores = ot.join()
    reps, pv = [], []
    k = 0
    for i, q in enumerate(reqs):
        nb = Bg if i in check_ids else 1
        gb = res[k:k + nb]
        k += nb
        for r in gb:
            assert r["n_escaped"] + r["n_absorbed"] + r["n_capped"] == r["n_emitted"]
        if i in check_ids:
            j = check_ids.index(i)
            ob = ores[j * Bo:(j + 1) * Bo]
            rep, p = compare(f"serving_req{i}_{q['geom']}_tau{q['tau0']:.3g}_T{q['T']:.3g}", gb, ob, cams=False)
            reps.append(rep)
            pv += p
    check(reps, pv)


def test_cfg5_cosmological_box(O, colt, ctx):
    """The synthetic cosmological box (9.4e6 leaves), five sources a step,
    three cameras of 512^2 x 256: GPU 48 steps and oracle 8 steps of 5 x 16
    packets, cameras at 16^2 blocks of 32^2 pixels; the 512^2 images of 5 x 32
    GPU packets pooled against their 16^2 tally."""
    import bench
    g, srcs, cams, cnb, label = bench.octree_workload("cosmo")
    Bg, Bo, n, blk = 48, 8, 16, 32
    nb = 512 // blk
    ns = len(srcs)

    def spec(j, m, off, npix):
        pos, sig = srcs[j]
        return S.RunSpec(n_packets=m, seed=300 + j, src_pos=pos, src_sigma=sig, albedo=0.32, spec_units=1,
                         spec_lo=-1000.0, spec_hi=1000.0, spec_nbins=200,
                         cameras=S.axis_cameras(npix, ("+x", "+y", "+z")), cam_units=1,
                         cam_lo=-1000.0, cam_hi=1000.0, cam_nbins=cnb, precision=1, pid_offset=off)
    ot = OracleThread(O, [(g, [spec(j, n, 10 ** 7 + b * n, nb) for b in range(Bo) for j in range(ns)], True)],
                      workers=8)
    h = colt.colt_create_grid(ctx, g)
    try:
        res = gpu_served(colt, ctx, [(h, spec(j, n, b * n, nb)) for b in range(Bg) for j in range(ns)], block_pix=1)
        pooled = pooling_check(colt, ctx, h, [(spec(j, 32, 5 * 10 ** 6, 512), spec(j, 32, 5 * 10 ** 6, nb))
                                              for j in range(ns)], blk)
    finally:
        colt.colt_destroy_grid(ctx, h)
    ores = ot.join()
    for i, r in enumerate(ores):
        r["blocks"] = oracle_blocks(r, spec(i % ns, n, 0, nb), nb)
    gb = [add_results(res[b * ns:(b + 1) * ns]) for b in range(Bg)]
    ob = [add_results(ores[b * ns:(b + 1) * ns]) for b in range(Bo)]
    rep, pv = compare(label, gb, ob, cams=True, images=True)
    rep["pooling_rel_l1"] = pooled
    assert rep["f_esc_gpu"] == 1.0 and rep["f_esc_oracle"] == 1.0        # no dust
    check([rep], pv)
