"""Pins of the oracle on octree grids (no GPU).

  * point location against a brute-force search over the leaf boxes with the
    half-open / direction tie rule;
  * an octree whose leaves are the cells of a 2^L Cartesian cube (in a
    shuffled order) reproduces the Cartesian walk packet by packet;
  * pure absorber on a mixed-level octree: each camera's emission peel-off is
    exactly exp(-tau) with tau summed over the leaf boxes the axis ray crosses
    (Sec. 6.1, Eq. SB; brute force over all leaves);
  * Eq. atauNL on mixed-level octrees of piecewise-uniform density: the path
    sums reduce to distances to the box edge or to the density jump.
"""
import numpy as np
import pytest

from paper_1409_4480_gb300 import synth as S

R = S.PC_CM


def _random_octree(seed, min_level=1, max_level=4, p=0.45):
    rng = np.random.default_rng(seed)
    lo, hi = np.array([-R] * 3), np.array([R] * 3)

    def refine(c, s, L):
        return rng.uniform(size=len(c)) < p

    return lo, hi, *S.octree_refine(lo, hi, refine, min_level, max_level)


def _boxes(lo, hi, lv, ijk):
    # leaf faces lo + i s_L with s_L = (hi - lo) 2^-L, one rounding each
    s = (hi - lo)[None, :] * np.exp2(-lv.astype(np.float64))[:, None]
    i = ijk.astype(np.float64)
    return lo[None, :] + i * s, lo[None, :] + (i + 1.0) * s


def test_refine_tiles_the_box():
    lo, hi, lv, ijk = _random_octree(1)
    _, s = S.leaf_geometry(lo, hi, lv, ijk)
    assert np.isclose(np.prod(s, axis=1).sum(), np.prod(hi - lo), rtol=1e-12)
    assert len(np.unique(np.c_[lv, ijk], axis=0)) == len(lv)
    assert lv.min() == 1 and lv.max() == 4


def test_octree_locate_brute_force(O):
    lo, hi, lv, ijk = _random_octree(2)
    g = S.octree_grid(lo, hi, lv, ijk, dict(n_HI=np.ones(len(lv)), T=np.full(len(lv), 1e4)))
    blo, bhi = _boxes(lo, hi, lv, ijk)
    rng = np.random.default_rng(3)
    # generic points, points on leaf faces / edges / vertices, and the box faces
    pts = list(rng.uniform(-R, R, (60, 3)))
    for i in rng.integers(0, len(lv), 40):
        q = rng.uniform(blo[i], bhi[i])
        pts.append(np.array([blo[i][0], q[1], q[2]]))
        pts.append(np.array([bhi[i][0], bhi[i][1], q[2]]))
        pts.append(blo[i].copy())
    pts += [np.array([-R, 0.1 * R, 0.2 * R]), np.array([R, 0.1 * R, 0.2 * R])]
    dirs = [np.array(d, float) for d in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                                         (0.6, -0.8, 0.0), (-0.48, 0.6, -0.64), (0.0, 0.0, 0.0)]]
    for p in pts:
        for d in dirs:
            inside = (p > blo) & (p < bhi)
            on_lo, on_hi = p == blo, p == bhi
            ok = np.all(inside | (on_lo & (d >= 0)) | (on_hi & (d < 0)), axis=1)
            want = np.flatnonzero(ok)
            assert len(want) <= 1
            got = O.octree_locate(g, p, d)
            assert got == (want[0] if len(want) else -1), (p, d)


def test_octree_of_cartesian_cube_matches_cartesian(O):
    gc = S.sphere(16, 1e4, 1e5, v_max_kms=80.0, tau_dust=0.7)
    go = S.octree_from_cartesian(gc, seed=5)
    spec = S.RunSpec(n_packets=600, seed=41, albedo=0.32, spec_units=1, spec_lo=-400, spec_hi=400, spec_nbins=80,
                     cameras=S.axis_cameras(0), cam_lo=-400, cam_hi=400, cam_nbins=40,
                     src_pos=(0.13 * R, -0.21 * R, 0.05 * R))
    rc = O.run(gc, spec, per_packet=True)
    ro = O.run(go, spec, per_packet=True)
    same = (rc["pk_status"] == ro["pk_status"]) & (rc["pk_nscat"] == ro["pk_nscat"]) & \
           (np.abs(rc["pk_freq"] - ro["pk_freq"]) <= 1e-9 * np.maximum(1.0, np.abs(rc["pk_freq"])))
    assert np.count_nonzero(same) >= 0.99 * len(same)
    # the non-local estimate is a property of the cells, whatever their order
    order = np.lexsort((go.leaf_ijk[:, 0], go.leaf_ijk[:, 1], go.leaf_ijk[:, 2]))
    assert np.allclose(O.atau_nl(go, 0.5)[order], O.atau_nl(gc, 0.5), rtol=1e-12, atol=0)


def _axis_tau(blo, bhi, kd, p, ax, sgn, lo, hi):
    """Optical depth from p to the box edge along +-axis through the leaf boxes."""
    t = [a for a in range(3) if a != ax]
    hit = np.all((blo[:, t] <= p[t]) & (p[t] < bhi[:, t]), axis=1)
    if sgn > 0:
        seg = np.clip(bhi[:, ax], p[ax], hi[ax]) - np.clip(blo[:, ax], p[ax], hi[ax])
    else:
        seg = np.clip(bhi[:, ax], lo[ax], p[ax]) - np.clip(blo[:, ax], lo[ax], p[ax])
    return float(np.sum(np.where(hit, kd * seg, 0.0)))


def test_octree_peel_attenuation_exact(O):
    lo, hi, lv, ijk = _random_octree(6, min_level=1, max_level=5, p=0.5)
    rng = np.random.default_rng(7)
    kd = rng.uniform(0.2, 3.0, len(lv)) / R
    g = S.octree_grid(lo, hi, lv, ijk, dict(n_HI=np.zeros(len(lv)), T=np.full(len(lv), 1e4), k_dust=kd))
    src = np.array([0.1234, -0.2345, 0.3456]) * R
    N = 200
    spec = S.RunSpec(n_packets=N, seed=8, albedo=0.0, spec_lo=-5, spec_hi=5, src_pos=tuple(src),
                     cameras=S.axis_cameras(0), cam_units=0, cam_lo=-5, cam_hi=5, cam_nbins=10)
    r = O.run(g, spec)
    blo, bhi = _boxes(lo, hi, lv, ijk)
    kd32 = g.k_dust.astype(np.float64)
    for cam, (ax, sgn) in enumerate([(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)]):
        tau = _axis_tau(blo, bhi, kd32, src, ax, sgn, lo, hi)
        assert r["cam_total"][cam] / N == pytest.approx(np.exp(-tau), rel=1e-9)


def test_octree_atau_nl_piecewise_uniform(O):
    lo, hi, lv, ijk = _random_octree(9, min_level=2, max_level=5, p=0.4)
    c, s = S.leaf_geometry(lo, hi, lv, ijk)
    blo, bhi = _boxes(lo, hi, lv, ijk)
    n = np.where(c[:, 0] > 0.0, 3.0, 1.0)          # a density jump at x = 0 (a face at every level >= 1)
    g = S.octree_grid(lo, hi, lv, ijk, dict(n_HI=n, T=np.full(len(lv), 1e4)))
    got = O.atau_nl(g, 0.5)
    ak = O.damping_a(1e4) * O.sigma0(1e4) * g.n_HI.astype(np.float64)
    left = c[:, 0] < 0.0
    # paths run through equal density to the box edge, or stop at the jump at x = 0
    d = np.stack([np.where(left, 0.0 - bhi[:, 0], hi[0] - bhi[:, 0]),
                  np.where(left, blo[:, 0] - lo[0], blo[:, 0] - 0.0),
                  hi[1] - bhi[:, 1], blo[:, 1] - lo[1], hi[2] - bhi[:, 2], blo[:, 2] - lo[2]], axis=1)
    want = ak * d.min(axis=1)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-300)
    assert np.count_nonzero(want == 0.0) > 0 and np.count_nonzero(want > 0.0) > 0
