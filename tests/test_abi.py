"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/colt.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "colt.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(colt_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("colt_create_grid", "colt_run", "colt_submit", "colt_poll", "colt_read_spectrum"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1409_4480_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (colt_\w+)", nm))
    assert set(_declared()) <= exported


def test_binding_covers_every_entry_point():
    from paper_1409_4480_gb300 import colt
    assert set(colt.EXPORTS) == set(_declared())
    for name in colt.EXPORTS:
        assert callable(getattr(colt, name))


def test_binding_struct_layout_matches_header():
    # compile a tiny host program that prints sizeof/offsetof of the ABI structs
    from paper_1409_4480_gb300 import colt
    src = os.path.join(ROOT, "tests", "pins", "abi_layout.c")
    exe = os.path.join(ROOT, "tests", "pins", f"abi_layout.{os.uname().machine}.bin")
    subprocess.run(["gcc", "-O0", "-I" + os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = dict(zip(out[0::2], map(int, out[1::2])))
    assert sizes["colt_grid_desc"] == ctypes.sizeof(colt.GridDesc)
    assert sizes["colt_camera"] == ctypes.sizeof(colt.Camera)
    assert sizes["colt_run_params"] == ctypes.sizeof(colt.RunParams)
    assert sizes["colt_result"] == ctypes.sizeof(colt.Result)
    assert sizes["colt_stats"] == ctypes.sizeof(colt.Stats)
    assert sizes["colt_launch_config"] == ctypes.sizeof(colt.LaunchConfig)
    assert sizes["colt_scatter_io"] == ctypes.sizeof(colt.ScatterIO)
    assert sizes["off_scatter_n_trials"] == colt.ScatterIO.n_trials.offset
    assert sizes["off_run_precision"] == colt.RunParams.precision.offset
    assert sizes["off_run_emission"] == colt.RunParams.emission.offset
    assert sizes["off_run_source"] == colt.RunParams.source.offset
    assert sizes["off_result_pk_freq"] == colt.Result.pk_freq.offset
    assert sizes["colt_source"] == ctypes.sizeof(colt.Source)
    assert sizes["off_run_sources"] == colt.RunParams.sources.offset
    assert sizes["off_stats_kernel_ms"] == colt.Stats.ctx_kernel_ms.offset
    assert sizes["off_stats_longest"] == colt.Stats.longest_history.offset
    assert sizes["off_stats_peel_visits"] == colt.Stats.ctx_peel_visits.offset
    assert sizes["off_launch_refill_min"] == colt.LaunchConfig.refill_min.offset


def test_no_cpu_fallback_in_product_path():
    # the product package must not import the oracle
    pkg = os.path.join(ROOT, "paper_1409_4480_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, f)) as fh:
                    txt = fh.read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f


def test_noalloc_binding_rejects_bad_buffers_before_calling():
    # colt_run_noalloc takes bare pointers and no lengths: the binding checks
    # every tensor first (these CPU tensors never reach the library)
    import pytest
    import torch
    from paper_1409_4480_gb300 import colt
    from paper_1409_4480_gb300 import synth as S
    g = S.uniform_box((4, 4, 4), (-1e18,) * 3, (1e18,) * 3, 1e-3, 1e4)
    spec = S.RunSpec(n_packets=10, seed=1, cameras=S.axis_cameras(0), cam_nbins=20)
    good = dict(spec=torch.zeros(spec.spec_nbins, dtype=torch.int64),
                counters=torch.zeros(8, dtype=torch.int64),
                cam_spec=torch.zeros((6, 20), dtype=torch.float64),
                cam_spec2=torch.zeros((6, 20), dtype=torch.float64))
    short = torch.zeros(g.n_cells * 8 - 1, dtype=torch.float32)
    with pytest.raises(ValueError, match="records.*elements"):
        colt.colt_run_noalloc([g], [short], [spec], [good])
    with pytest.raises(ValueError, match="dtype"):
        colt.colt_run_noalloc([g], [torch.zeros(g.n_cells * 8, dtype=torch.float64)], [spec], [good])
    with pytest.raises(ValueError, match="cam_spec2.*elements"):
        colt.colt_run_noalloc([g], [torch.zeros(g.n_cells * 8)], [spec],
                              [{**good, "cam_spec2": torch.zeros(6 * 20 - 1, dtype=torch.float64)}])
    with pytest.raises(ValueError, match="counters"):
        colt.colt_run_noalloc([g], [torch.zeros(g.n_cells * 8)], [spec], [{**good, "counters": None}])
    with pytest.raises(ValueError, match="not a CUDA tensor"):
        colt.colt_run_noalloc([g], [torch.zeros(g.n_cells * 8)], [spec], [good])
