"""Failure detection without faulting the GPU: bounded waits that run out,
the kernel's error flag raised by bad device inputs, cancelling requests.

None of these faults, traps or hangs the device: the wait that runs out is
the host's (colt_wait), the bad input is non-finite cell records that the
kernel detects when a packet leaves the box (no index is derived from a
record, so nothing is accessed out of range), and cancelling only stops
packets from being handed out."""
import numpy as np
import pytest

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(colt):
    c = colt.colt_init(0)
    yield c
    colt.colt_finalize(c)


def _long_request(n=400000):
    # a thick dusty sphere: long enough that a 1 ms wait cannot see it finish
    return S.sphere(48, 1e4, 1e7, tau_dust=0.5), S.RunSpec(
        n_packets=n, seed=21, albedo=0.32, spec_units=1, spec_lo=-800, spec_hi=800, spec_nbins=80)


def test_wait_times_out_and_the_request_still_completes(colt, ctx):
    g, spec = _long_request()
    h = colt.colt_create_grid(ctx, g)
    try:
        rid = colt.colt_submit(ctx, h, spec)
        with pytest.raises(colt.ColtError) as e:
            colt.colt_wait(ctx, rid, 1.0)
        assert e.value.code == colt.COLT_ETIMEOUT
        colt.colt_wait(ctx, rid, -1.0)                 # no limit: finishes
        st = colt.colt_poll(ctx, rid)
        assert st["done"] and not st["cancelled"] and st["packets_done"] == spec.n_packets
        r = colt.colt_read_result(ctx, rid, spec)
        assert r["n_emitted"] == spec.n_packets
        assert r["n_escaped"] + r["n_absorbed"] + r["n_capped"] == spec.n_packets
        # the result equals the blocking solve of the same request
        ref = colt.colt_run(ctx, h, spec)
        assert np.array_equal(r["spec"], ref["spec"]) and r["n_scat"] == ref["n_scat"]
        colt.colt_release(ctx, rid)
    finally:
        colt.colt_destroy_grid(ctx, h)


def test_non_finite_device_records_raise_the_device_error(colt):
    # colt_run_noalloc takes device cell records that the host never checks;
    # NaN records make every packet leave with a non-finite frequency, which
    # the kernel reports through its error flag (COLT_EDEVICE) instead of
    # tallying; the context stays usable
    import torch
    g = S.sphere(16, 1e4, 1e4, tau_dust=0.3)
    spec = S.RunSpec(n_packets=2000, seed=5, albedo=0.32, spec_units=1, spec_lo=-300, spec_hi=300, spec_nbins=30)
    c = colt.colt_init(0)
    try:
        h = colt.colt_create_grid(c, g)
        good = torch.from_numpy(colt.colt_read_cells(c, h, g.n_cells)).cuda().reshape(-1)
        colt.colt_destroy_grid(c, h)
    finally:
        colt.colt_finalize(c)
    bad = torch.full_like(good, float("nan"))
    t = dict(spec=torch.zeros(spec.spec_nbins, dtype=torch.int64, device="cuda"),
             counters=torch.zeros(8, dtype=torch.int64, device="cuda"))
    assert colt.colt_run_noalloc([g], [bad], [spec], [t]) == colt.COLT_EDEVICE
    torch.cuda.synchronize()
    cnt = t["counters"].cpu().numpy()
    assert cnt[0] == 2000 and cnt[1] == 0 and cnt[3] == 2000   # all ended as capped, none tallied
    assert int(t["spec"].sum()) == 0
    # the same call on valid records succeeds afterwards
    assert colt.colt_run_noalloc([g], [good], [spec], [t]) == colt.COLT_OK
    torch.cuda.synchronize()
    cnt = t["counters"].cpu().numpy()
    assert cnt[0] == 2000 and cnt[1] + cnt[2] + cnt[3] == 2000 and cnt[3] == 0


def test_cancel_running_and_queued_requests(colt, ctx):
    g, spec = _long_request(8 << 20)     # more packets than the six serving launches (2^20 each) take
    h = colt.colt_create_grid(ctx, g)
    try:
        rid = colt.colt_submit(ctx, h, spec)
        colt.colt_cancel(ctx, rid)
        colt.colt_wait(ctx, rid, -1.0)
        st = colt.colt_poll(ctx, rid)
        assert st["done"] and st["cancelled"]
        assert 0 < st["packets_done"] < spec.n_packets   # the launches already under way finished
        r = colt.colt_read_result(ctx, rid, spec)
        assert r["n_emitted"] == st["packets_done"]
        assert r["n_escaped"] + r["n_absorbed"] + r["n_capped"] == r["n_emitted"]
        colt.colt_release(ctx, rid)
        # a small request behind two large ones (which hold every launch
        # slot): cancelled before it starts, it is done with empty results
        small = S.RunSpec(**{**spec.__dict__, "n_packets": 1000})
        ids = [colt.colt_submit(ctx, h, spec) for _ in range(2)]
        q = colt.colt_submit(ctx, h, small)
        colt.colt_cancel(ctx, q)
        colt.colt_wait(ctx, q, -1.0)
        st = colt.colt_poll(ctx, q)
        assert st["done"] and st["cancelled"] and st["packets_done"] <= 1000
        if st["packets_done"] == 0:
            r = colt.colt_read_result(ctx, q, small)
            assert r["n_emitted"] == 0 and int(r["spec"].sum()) == 0
        for i in ids:
            colt.colt_cancel(ctx, i)
        for i in ids + [q]:
            colt.colt_wait(ctx, i, -1.0)
            colt.colt_release(ctx, i)
        # releasing a running request is refused until it is done
        rid = colt.colt_submit(ctx, h, spec)
        with pytest.raises(colt.ColtError) as e:
            colt.colt_release(ctx, rid)
        assert e.value.code == colt.COLT_EAGAIN
        colt.colt_cancel(ctx, rid)
        colt.colt_wait(ctx, rid, -1.0)
        colt.colt_release(ctx, rid)
    finally:
        colt.colt_destroy_grid(ctx, h)
