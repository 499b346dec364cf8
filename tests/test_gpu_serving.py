"""Serving through the C ABI: colt_submit / colt_poll / colt_wait /
colt_read_spectrum / colt_read_image with continuous batching.  Each request's result in the mix
equals its result alone (colt_run with the same grid and parameters):
integer tallies bitwise, peel-off sums up to FP64 summation order.  Memory
admission queues what does not fit and rejects what never can."""

import time

import numpy as np
import pytest

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _mix():
    grids = [S.sphere(24, 1e4, 1e4, v_max_kms=100.0, tau_dust=0.5),
             S.slab(16, 100.0, 1e5, v_max_kms=-50.0, tau_dust=0.2, nxy=4),
             S.sphere(16, 10.0, 3e4)]
    cams = S.axis_cameras(0)
    cams[0] = S.Camera(cams[0].direction, 8)      # one camera with an 8 x 8 image
    reqs = []
    for i, (gi, n) in enumerate([(0, 3000), (1, 20000), (2, 1000), (0, 50000), (1, 700), (2, 9000)]):
        reqs.append((gi, S.RunSpec(n_packets=n, seed=4000 + i, albedo=0.32, spec_units=1, spec_lo=-400,
                                   spec_hi=400, spec_nbins=80, cameras=cams if i % 2 == 0 else [],
                                   cam_units=1, cam_lo=-400, cam_hi=400, cam_nbins=40)))
    return grids, reqs


def test_batched_equals_alone(colt):
    ctx = colt.colt_init(0)
    try:
        grids, reqs = _mix()
        hs = [colt.colt_create_grid(ctx, g) for g in grids]
        alone = [colt.colt_run(ctx, hs[gi], sp, images=bool(sp.cameras)) for gi, sp in reqs]
        ids = []
        image_flux = 0.0
        for gi, sp in reqs:                      # arrivals while earlier work runs
            ids.append(colt.colt_submit(ctx, hs[gi], sp))
            colt.colt_poll(ctx, ids[-1])
        for rid in ids:
            colt.colt_wait(ctx, rid, timeout_ms=120000)
        for rid, (gi, sp), ref in zip(ids, reqs, alone):
            st = colt.colt_poll(ctx, rid)
            assert st["done"] and st["packets_done"] == sp.n_packets and st["latency_ms"] > 0
            got = colt.colt_read_result(ctx, rid, sp)
            assert np.array_equal(got["spec"], ref["spec"])
            for key in ("n_emitted", "n_escaped", "n_absorbed", "n_capped", "n_scat", "n_scat_hi"):
                assert got[key] == ref[key], key
            if sp.cameras:
                assert np.allclose(got["cam_spec"], ref["cam_spec"], rtol=1e-9, atol=1e-300)
                c0 = colt.colt_read_spectrum(ctx, rid, 0, sp.cam_nbins)
                assert np.allclose(c0, ref["cam_spec"][0], rtol=1e-9, atol=1e-300)
                img = colt.colt_read_image(ctx, rid, 0, 8, sp.cam_nbins)
                assert np.allclose(img.ravel(), ref["cam_image"][: img.size], rtol=1e-9, atol=1e-300)
                # the image plane spans the box: every +x contribution lands in it
                # (none on the periodic slab, whose x axis has no observer)
                assert img.sum() == pytest.approx(ref["cam_spec"][0].sum(), rel=1e-9, abs=1e-300)
                image_flux += img.sum()
                with pytest.raises(colt.ColtError):
                    colt.colt_read_image(ctx, rid, 1, 8, sp.cam_nbins)     # camera 1 has no image
            esc = colt.colt_read_spectrum(ctx, rid, -1, sp.spec_nbins)
            assert np.array_equal(esc, ref["spec"].astype(np.float64))
            colt.colt_release(ctx, rid)
        assert image_flux > 0
        for h in hs:
            colt.colt_destroy_grid(ctx, h)
    finally:
        colt.colt_finalize(ctx)


def test_submit_many_shares_one_launch_and_equals_alone(colt):
    # a batch submitted together is scheduled together: the six requests of
    # the mix (83 700 packets, one precision, Cartesian grids) go into one
    # launch, where colt_submit would start the first ones in launch slots of
    # their own; each result still equals the request's solve alone
    ctx = colt.colt_init(0)
    try:
        grids, reqs = _mix()
        hs = [colt.colt_create_grid(ctx, g) for g in grids]
        alone = [colt.colt_run(ctx, hs[gi], sp, images=bool(sp.cameras)) for gi, sp in reqs]
        z = colt.colt_submit(ctx, hs[0], S.RunSpec(n_packets=0, seed=0))     # done at once, launches nothing
        st0 = colt.colt_poll(ctx, z)
        launches0 = st0["launches"]
        colt.colt_release(ctx, z)
        ids = colt.colt_submit_many(ctx, [(hs[gi], sp) for gi, sp in reqs])
        assert len(ids) == len(reqs) and ids == sorted(ids)
        for rid in ids:
            colt.colt_wait(ctx, rid, timeout_ms=120000)
        assert colt.colt_poll(ctx, ids[0])["launches"] == launches0 + 1
        # the longest history is known once the launch has ended (a request
        # can be done before that): poll until it is, then it lies between
        # the mean scatterings per packet and the request's total
        deadline = time.time() + 60.0
        while colt.colt_poll(ctx, ids[0])["longest_history"] == 0 and time.time() < deadline:
            time.sleep(0.01)
        # the context's visit totals grew by the launch's: flight visits are
        # those of the same packets alone, peel-off visits nearly so
        st1 = colt.colt_poll(ctx, ids[0])
        assert st1["cell_visits"] - st0["cell_visits"] == sum(r["n_cell_visits"] for r in alone)
        pv = sum(r["n_peel_visits"] for r in alone)
        assert pv > 0 and abs(st1["peel_visits"] - st0["peel_visits"] - pv) <= 1e-3 * pv
        for rid, (gi, sp), ref in zip(ids, reqs, alone):
            st = colt.colt_poll(ctx, rid)
            assert st["done"] and st["packets_done"] == sp.n_packets
            assert ref["n_scat"] / sp.n_packets <= st["longest_history"] <= ref["n_scat"]
            got = colt.colt_read_result(ctx, rid, sp)
            assert np.array_equal(got["spec"], ref["spec"])
            for key in ("n_emitted", "n_escaped", "n_absorbed", "n_capped", "n_scat", "n_scat_hi"):
                assert got[key] == ref[key], key
            if sp.cameras:
                assert np.allclose(got["cam_spec"], ref["cam_spec"], rtol=1e-9, atol=1e-300)
                img = colt.colt_read_image(ctx, rid, 0, 8, sp.cam_nbins)
                assert np.allclose(img.ravel(), ref["cam_image"][: img.size], rtol=1e-9, atol=1e-300)
            colt.colt_release(ctx, rid)
        # all or none: a batch with an unknown grid queues nothing
        z1 = colt.colt_submit(ctx, hs[0], S.RunSpec(n_packets=0, seed=0))
        with pytest.raises(colt.ColtError) as e:
            colt.colt_submit_many(ctx, [(hs[0], reqs[0][1]), (hs[-1] + 1000, reqs[0][1])])
        assert e.value.code == colt.COLT_ENOTFOUND
        z2 = colt.colt_submit(ctx, hs[0], S.RunSpec(n_packets=0, seed=0))
        assert z2 == z1 + 1
        assert colt.colt_poll(ctx, z2)["launches"] == launches0 + 1
        for q in (z1, z2):
            colt.colt_release(ctx, q)
        assert colt.colt_submit_many(ctx, []) == []
        for h in hs:
            colt.colt_destroy_grid(ctx, h)
    finally:
        colt.colt_finalize(ctx)


def test_admission_by_memory(colt):
    g = S.sphere(16, 1e4, 1e4)
    grid_bytes = g.n_cells * 32
    big = S.RunSpec(n_packets=2000, seed=1, spec_units=1, spec_lo=-400, spec_hi=400, spec_nbins=100,
                    cameras=S.axis_cameras(64), cam_units=1, cam_lo=-400, cam_hi=400, cam_nbins=100)
    img_bytes = 6 * 64 * 64 * 100 * 8
    ctx = colt.colt_init(0, mem_budget_bytes=grid_bytes + int(1.5 * img_bytes) + (1 << 20))
    try:
        h = colt.colt_create_grid(ctx, g)
        # images are not kept by serving requests; make requests heavy through bins
        heavy = S.RunSpec(**{**big.__dict__, "cam_nbins": 40000, "cameras": S.axis_cameras(0)})
        r1 = colt.colt_submit(ctx, h, heavy)
        r2 = colt.colt_submit(ctx, h, S.RunSpec(**{**heavy.__dict__, "seed": 2}))
        st2 = colt.colt_poll(ctx, r2)
        colt.colt_wait(ctx, r1, timeout_ms=60000)
        colt.colt_release(ctx, r1)               # frees memory -> r2 admitted
        colt.colt_wait(ctx, r2, timeout_ms=60000)
        assert colt.colt_poll(ctx, r2)["done"]
        colt.colt_release(ctx, r2)
        # a request that can never fit is refused at once
        never = S.RunSpec(**{**heavy.__dict__, "cam_nbins": 4_000_000})
        with pytest.raises(colt.ColtError) as e:
            colt.colt_submit(ctx, h, never)
        assert e.value.code == colt.COLT_ENOMEM
        # reading a result before completion is EAGAIN
        r3 = colt.colt_submit(ctx, h, S.RunSpec(n_packets=200000, seed=3, spec_lo=-40, spec_hi=40))
        st = colt.colt_poll(ctx, r3)
        if not st["done"]:
            with pytest.raises(colt.ColtError) as e:
                colt.colt_read_spectrum(ctx, r3, -1, 100)
            assert e.value.code == colt.COLT_EAGAIN
        colt.colt_wait(ctx, r3, timeout_ms=120000)
        colt.colt_release(ctx, r3)
        colt.colt_destroy_grid(ctx, h)
        del st2
    finally:
        colt.colt_finalize(ctx)


def test_autotune_keeps_results(colt):
    # the launch configuration changes only the speed: integer tallies are
    # bitwise the same under the tuned configuration, blocking and served
    ctx = colt.colt_init(0)
    try:
        g = S.sphere(24, 1e4, 1e5, v_max_kms=100.0, tau_dust=0.5)
        h = colt.colt_create_grid(ctx, g)
        sp = S.RunSpec(n_packets=20000, seed=4321, albedo=0.32, spec_units=1, spec_lo=-600, spec_hi=600,
                       spec_nbins=60, cameras=S.axis_cameras(0), cam_lo=-600, cam_hi=600, cam_nbins=30)
        before = colt.colt_run(ctx, h, sp)
        cfg = colt.colt_autotune(ctx, h, sp)
        assert cfg["variant"] in (0, 1, 2) and cfg["blocks_per_sm"] >= 1 and cfg["scatterings_per_s"] > 0
        assert cfg["warps_per_block"] in (4, 8, 16) and cfg["refill_min"] in (1, 4, 12)
        # every block size and refill threshold gives the same results
        for w, m in ((4, 1), (16, 12), (8, 32)):
            colt.colt_set_launch_config(ctx, colt.COLT_MIXED, colt.COLT_CARTESIAN, 0, 0, w, m)
            r = colt.colt_run(ctx, h, sp)
            assert np.array_equal(r["spec"], before["spec"]) and r["n_scat"] == before["n_scat"]
        with pytest.raises(colt.ColtError):
            colt.colt_set_launch_config(ctx, colt.COLT_PLAIN, colt.COLT_CARTESIAN, 0, 0, 16, 1)   # FP64: 8 warps only
        colt.colt_set_launch_config(ctx, colt.COLT_MIXED, colt.COLT_CARTESIAN, cfg["variant"], cfg["blocks_per_sm"],
                                    cfg["warps_per_block"], cfg["refill_min"])
        after = colt.colt_run(ctx, h, sp)
        rid = colt.colt_submit(ctx, h, sp)
        colt.colt_wait(ctx, rid, timeout_ms=120000)
        served = colt.colt_read_result(ctx, rid, sp)
        colt.colt_release(ctx, rid)
        for r in (after, served):
            assert np.array_equal(r["spec"], before["spec"])
            assert r["n_scat"] == before["n_scat"] and r["n_escaped"] == before["n_escaped"]
            assert np.allclose(r["cam_spec"], before["cam_spec"], rtol=1e-9, atol=1e-300)
        sp64 = S.RunSpec(**{**sp.__dict__, "precision": 0, "n_packets": 3000})
        cfg64 = colt.colt_autotune(ctx, h, sp64)
        assert cfg64["variant"] == 0
        colt.colt_destroy_grid(ctx, h)
    finally:
        colt.colt_finalize(ctx)
