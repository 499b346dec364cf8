"""Host-side logic of the benchmark (no GPU): workload definitions, the
flux-table observables, and the rule that the reported DRAM traffic comes
only from a capture of the current kernel sources."""
import hashlib
import os

import numpy as np
import pytest

import bench


def test_sphere_suite_cases():
    cs = bench.cases()
    assert len(cs) == 9 and len(set(cs)) == 9
    assert {t for t, _ in cs} == {1e5, 1e6, 1e7} and {v for _, v in cs} == {-200.0, 0.0, 200.0}
    sp = bench.case_spec(4, 1000, 7000)
    assert sp.n_packets == 1000 and sp.pid_offset == 7000 and sp.seed == 204 and len(sp.cameras) == 6


def test_serving_requests_are_seeded_and_in_range():
    a, b = bench.serving_requests(64), bench.serving_requests(64)
    assert a == b
    for r in a:
        assert r["geom"] in ("sphere", "slab")
        assert 1e4 <= r["tau0"] <= 1e8 and 10.0 <= r["T"] <= 1e5
        assert -300.0 <= r["v"] <= 300.0 and 0.0 <= r["td"] <= 2.0
        assert 1e4 <= r["n"] <= 1e6 and r["w"] > 0


def test_slab_suite_columns():
    suite = bench.slab_suite()
    fixed_tau = [t for k, _, t in suite if k == "tau0"]
    assert fixed_tau == [1e7] * 5
    # fixed column N_H = 1.7e20 cm^-2: tau0 = N_H sigma_0(T) = 1e7 T4^-1/2
    for k, T, t in suite:
        if k == "column":
            assert t == pytest.approx(1.7e20 * 5.898e-14 / np.sqrt(T / 1e4), rel=0.01)


def test_galaxy_models_and_observables():
    assert len(bench.GALAXY_MODELS) == 16 and len(set(bench.GALAXY_MODELS)) == 16
    nb = 10
    cs = np.zeros((6, nb))
    cs[0:4, :] = 1.0                       # edge-on cameras: flat, 1 per bin
    cs[4:6, nb // 2:] = 3.0                # face-on cameras: only red, 3 per bin
    spec = np.full(nb, 1.0)
    o = bench.galaxy_observables({"cam_spec": cs, "spec": spec, "n_escaped": 10, "n_emitted": 10})
    assert o["F/F_Omega_xy"] == pytest.approx(1.0)
    assert o["F/F_Omega_z"] == pytest.approx(1.5)
    assert o["Fr/Fb_xy"] == pytest.approx(1.0) and o["Fr/Fb_Omega"] == pytest.approx(1.0)
    assert o["Fr/Fb_z"] > 1e10 and o["f_esc"] == 1.0


def test_traffic_only_from_a_capture_of_the_current_kernel(tmp_path, monkeypatch):
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(bench.ROOT, f), "rb") as fh:
            h.update(fh.read())
    good = tmp_path / "good.md"
    good.write_text(f"kernel_source_sha256: `{h.hexdigest()}`\ndram_bytes_per_unit: 0.5\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(good))
    assert bench.dram_bytes_per_scattering() == pytest.approx(0.5)
    stale = tmp_path / "stale.md"
    stale.write_text("kernel_source_sha256: `" + "0" * 64 + "`\ndram_bytes_per_unit: 0.5\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(stale))
    assert bench.dram_bytes_per_scattering() is None
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(tmp_path / "missing.md"))
    assert bench.dram_bytes_per_scattering() is None
