"""Host-side logic of the benchmark (no GPU): workload definitions, the
flux-table observables, and the rule that the roofline figures come
only from a capture of the current kernel sources."""
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


def test_roofline_only_from_a_capture_of_the_current_kernel(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    (tmp_path / "k_transport_good.md").write_text(
        f"kernel_source_sha256: `{h}`\nfp32_flop_per_scattering: 600\ndram_bytes_per_scattering: 0.5\n")
    (tmp_path / "k_transport_stale.md").write_text(
        "kernel_source_sha256: `" + "0" * 64 + "`\nfp32_flop_per_scattering: 600\ndram_bytes_per_scattering: 0.5\n")
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    u = bench.profile_units("good")
    assert u["fp32_flop_per_scattering"] == 600 and u["dram_bytes_per_scattering"] == 0.5
    assert bench.profile_units("stale") is None and bench.profile_units("missing") is None
    info = {"sm_count": 152}
    r = bench.roofline(u, scat=1e9, kernel_ms=1000.0, served_rate=2e9, info=info)
    peak = 152 * 128 * 2 * bench.measured_peaks().get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(600 * 1e9 / 1.0 / 1e12)        # FP32 operations of the launch / its time
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] == pytest.approx(0.5 * 1e9)
    assert r["frac_served"] == pytest.approx(600 * 2e9 / 1e12 / peak)
    n = bench.roofline(None, 1e9, 1000.0, 2e9, info)
    assert n["achieved"] is None and n["traffic"] is None


def test_roofline_scales_the_capture_to_the_timed_work_mix(tmp_path, monkeypatch):
    # a capture with cameras (600 FP32 operations per scattering at 20 peel-off
    # visits per scattering) and the same solves without them (200): the
    # per-scattering count follows the timed region's peel-off visits
    h = bench.kernel_source_hash()
    (tmp_path / "k_transport_w.md").write_text(
        f"kernel_source_sha256: `{h}`\nfp32_flop_per_scattering: 600\ndram_bytes_per_scattering: 0.5\n"
        "Launch: 1000 scatterings, 1100 flight cell visits, 20000 peel-off visits (900 rays)\n")
    (tmp_path / "k_transport_w_nocam.md").write_text(
        f"kernel_source_sha256: `{h}`\nfp32_flop_per_scattering_no_cameras: 200\n")
    (tmp_path / "k_transport_v.md").write_text((tmp_path / "k_transport_w.md").read_text())
    (tmp_path / "k_transport_v_nocam.md").write_text(
        "kernel_source_sha256: `" + "0" * 64 + "`\nfp32_flop_per_scattering_no_cameras: 200\n")
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    u = bench.profile_units("w")
    assert u["visits_per_scattering"] == {"cell": 1.1, "peel": 20.0}
    assert u["fp32_flop_per_scattering_no_cameras"] == 200
    info = {"sm_count": 152}
    def f(units, peel):
        return bench.roofline(units, 1e9, 1000.0, 2e9, info, mix={"cell": 1.0, "peel": peel})["flop_per_scattering"]
    assert f(u, 20.0) == pytest.approx(600)      # the capture's own mix: its count
    assert f(u, 0.0) == pytest.approx(200)       # no peel-off: the count without cameras
    assert f(u, 5.0) == pytest.approx(300)       # a quarter of the capture's peel-off visits
    assert bench.roofline(u, 1e9, 1000.0, 2e9, info)["flop_per_scattering"] == 600   # no mix given
    v = bench.profile_units("v")                 # a stale capture without cameras is not used
    assert "fp32_flop_per_scattering_no_cameras" not in v and f(v, 5.0) == pytest.approx(600)


def test_cosmo_step_specs_disjoint_ids():
    srcs = [((float(i), 0.0, 0.0), 0.0) for i in range(5)]
    a = bench.cosmo_specs(srcs, [], 256, 100, 0)
    b = bench.cosmo_specs(srcs, [], 256, 100, 500)
    ids = [(sp.seed, sp.pid_offset + k) for sp in a + b for k in range(sp.n_packets)]
    assert len(ids) == len(set(ids)) and len(a) == 5 and all(sp.n_packets == 100 for sp in a)
    assert [sp.seed for sp in a] == [300, 301, 302, 303, 304]
