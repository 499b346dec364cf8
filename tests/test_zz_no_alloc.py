"""colt_run_noalloc: the solve for callers that cannot allocate device memory
(code under another allocator's memory budget, or a library that must not
call cudaMalloc for its user).  The caller owns the cell records and the
tallies; the entry point keeps its launch header and counters in a static
device array.  Its results must equal colt_run's on the same grid and
parameters -- integer tallies exactly, peel-off sums up to FP64 summation
order -- on two calls in a row (the shared array is reused), and the second
call must leave the device's free memory unchanged.

This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1409_4480_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_noalloc_matches_colt_run_twice(colt):
    import torch
    g = S.sphere(24, 1e4, 1e4, v_max_kms=100.0, tau_dust=0.5)
    spec = S.RunSpec(n_packets=6000, seed=77, albedo=0.32, spec_units=1, spec_lo=-400, spec_hi=400,
                     spec_nbins=80, cameras=S.axis_cameras(8), cam_units=1, cam_lo=-400, cam_hi=400,
                     cam_nbins=40)
    ctx = colt.colt_init(0)
    try:
        h = colt.colt_create_grid(ctx, g)
        ref = colt.colt_run(ctx, h, spec, images=True)
        rec = torch.from_numpy(colt.colt_read_cells(ctx, h, g.n_cells)).cuda()
        colt.colt_destroy_grid(ctx, h)
    finally:
        colt.colt_finalize(ctx)
    dev = torch.device("cuda")
    t = dict(spec=torch.full((spec.spec_nbins,), 7, dtype=torch.int64, device=dev),
             counters=torch.full((8,), 7, dtype=torch.int64, device=dev),
             cam_spec=torch.ones((6, spec.cam_nbins), dtype=torch.float64, device=dev),
             cam_spec2=torch.ones((6, spec.cam_nbins), dtype=torch.float64, device=dev),
             cam_image=torch.ones((6 * 8 * 8 * spec.cam_nbins,), dtype=torch.float64, device=dev))
    for call in range(2):
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        rc = colt.colt_run_noalloc([g], [rec], [spec], [t], images=True)
        assert rc == colt.COLT_OK
        torch.cuda.synchronize()
        if call == 1:
            # after the first call (module loading, launch resources), a call
            # takes no device memory: the driver's free bytes and torch's
            # allocator both stay where they were
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        cnt = t["counters"].cpu().numpy().astype(np.uint64)
        assert cnt[0] == ref["n_emitted"] == 6000
        assert (cnt[1], cnt[2], cnt[3]) == (ref["n_escaped"], ref["n_absorbed"], ref["n_capped"])
        assert (cnt[4], cnt[5]) == (ref["n_scat"], ref["n_scat_hi"])
        assert np.array_equal(t["spec"].cpu().numpy().astype(np.uint64), ref["spec"])
        assert np.allclose(t["cam_spec"].cpu().numpy(), ref["cam_spec"], rtol=1e-9, atol=1e-300)
        assert np.allclose(t["cam_spec2"].cpu().numpy(), ref["cam_spec2"], rtol=1e-9, atol=1e-300)
        assert np.allclose(t["cam_image"].cpu().numpy(), ref["cam_image"], rtol=1e-9, atol=1e-300)


def test_noalloc_rejects_sizes_beyond_its_table(colt):
    import torch
    g = S.uniform_box((2, 2, 2), (-1e18, -1e18, -1e18), (1e18, 1e18, 1e18), 1e-3, 1e4)
    rec = torch.zeros(g.n_cells * 8, dtype=torch.float32, device="cuda")
    spec = S.RunSpec(n_packets=10, seed=1)
    t = dict(spec=torch.zeros(spec.spec_nbins, dtype=torch.int64, device="cuda"),
             counters=torch.zeros(8, dtype=torch.int64, device="cuda"))
    assert colt.colt_run_noalloc([g] * 9, [rec] * 9, [spec] * 9, [t] * 9) == colt.COLT_EINVAL
