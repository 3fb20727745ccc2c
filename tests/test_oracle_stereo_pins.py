"""Pins of the oracle's stereo triangulation gate (no GPU).

Each pin is fixed by geometry, not by the oracle's own formulas: exact
correspondences of known 3-D points must triangulate back to those points
with zero reprojection error; a rectified pair has depth f b / d; a pure
rotation has zero disparity everywhere; in a rectified pair every 3-D point
projects to equal rows, so a vertical misalignment e splits into two
reprojection errors that sum to at least e.
"""

import numpy as np

from oracle import stereo as S


def _rot(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rz = np.array([[cc, -sc, 0], [sc, cc, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _observe(K, X):
    """Pixel of 3-D point X (camera frame) under pinhole K = (fx, fy, cx, cy)."""
    fx, fy, cx, cy = K
    return np.stack([fx * X[:, 0] / X[:, 2] + cx, fy * X[:, 1] / X[:, 2] + cy], axis=1)


def _general_rig(seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    R = _rot(*rng.uniform(-0.08, 0.08, 3))
    t = np.array([-0.12, 0.004, -0.01]) + rng.uniform(-0.002, 0.002, 3)
    return S.Rig(kl=(458.0, 457.0, 367.5, 248.0), kr=(461.0, 460.0, 379.0, 255.5), R=R, t=t), rng


def test_exact_correspondences_recover_the_point():
    rig, rng = _general_rig()
    XL = np.stack([rng.uniform(-2, 2, 400), rng.uniform(-1.5, 1.5, 400), rng.uniform(1.0, 20.0, 400)], axis=1)
    XR = XL @ rig.R.T + rig.t
    # float64 observations: this pin is about the geometry, not input rounding
    pl, pr = _observe(rig.kl, XL), _observe(rig.kr, XR)
    xl = np.stack([(pl[:, 0] - rig.kl[2]) / rig.kl[0], (pl[:, 1] - rig.kl[3]) / rig.kl[1]], 1)
    xr = np.stack([(pr[:, 0] - rig.kr[2]) / rig.kr[0], (pr[:, 1] - rig.kr[3]) / rig.kr[1]], 1)
    Xh = S.triangulate_dlt(xl, xr, rig.R, rig.t)
    X = Xh[:, :3] / Xh[:, 3:]
    np.testing.assert_allclose(X, XL, rtol=1e-9)
    # through the gate (float32 observations): kept, tiny reprojection error
    r = S.stereo_gate(pl.astype(np.float32), pr.astype(np.float32), None, rig, S.GateParams(min_disp=0.5))
    assert (r.status == 1).all(), np.unique(r.reason, return_counts=True)
    assert np.maximum(r.e_left, r.e_right).max() < 1e-3
    np.testing.assert_allclose(r.xyz, XL, rtol=2e-3)
    np.testing.assert_allclose(r.z_right, XR[:, 2], rtol=2e-3)


def test_rectified_pair_depth_is_f_b_over_d():
    f, b = 460.0, 0.11
    rig = S.Rig(kl=(f, f, 375.5, 239.5), kr=(f, f, 375.5, 239.5), R=np.eye(3), t=np.array([-b, 0.0, 0.0]))
    ul = np.array([100.0, 300.0, 375.5, 600.0, 700.0])
    v = np.array([50.0, 239.5, 300.0, 400.0, 10.0])
    d = np.array([1.5, 4.0, 12.25, 30.0, 64.0])
    r = S.stereo_gate(np.stack([ul, v], 1), np.stack([ul - d, v], 1), None, rig, S.GateParams())
    assert (r.status == 1).all()
    np.testing.assert_allclose(r.disparity, d, rtol=1e-12)
    np.testing.assert_allclose(r.xyz[:, 2], f * b / d, rtol=1e-10)
    np.testing.assert_allclose(r.xyz[:, 0], (ul - 375.5) * (b / d), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r.xyz[:, 1], (v - 239.5) * (b / d), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r.z_right, r.z_left, rtol=1e-12)
    assert np.maximum(r.e_left, r.e_right).max() < 1e-9


def test_pure_rotation_has_no_disparity():
    rig, rng = _general_rig(3)
    rig.t = np.zeros(3)
    XL = np.stack([rng.uniform(-2, 2, 100), rng.uniform(-1.5, 1.5, 100), rng.uniform(1.0, 20.0, 100)], axis=1)
    pl, pr = _observe(rig.kl, XL), _observe(rig.kr, XL @ rig.R.T)
    r = S.stereo_gate(pl, pr, None, rig, S.GateParams(min_disp=0.01))
    assert r.disparity.max() < 1e-3
    assert (r.reason == S.GATE_DISP).all()


def test_far_point_and_negative_disparity():
    f, b = 460.0, 0.11
    rig = S.Rig(kl=(f, f, 375.5, 239.5), kr=(f, f, 375.5, 239.5), R=np.eye(3), t=np.array([-b, 0.0, 0.0]))
    pl = np.array([[300.0, 200.0], [300.0, 200.0], [300.0, 200.0], [300.0, 200.0]])
    # disparity 0.875 (below 1 px; 58 m), 1.25 (kept: 40 m), 0.5 (101 m), -3 (the distance is
    # 3 px, but the point triangulates behind the cameras)
    pr = pl - np.array([[0.875, 0], [1.25, 0], [0.5, 0], [-3.0, 0]])
    r = S.stereo_gate(pl, pr, None, rig, S.GateParams(min_disp=1.0))
    assert list(r.reason) == [S.GATE_DISP, S.GATE_OK, S.GATE_DISP, S.GATE_DEPTH]
    r = S.stereo_gate(pl, pr, None, rig, S.GateParams(min_disp=0.25, z_max=60.0))
    assert list(r.reason) == [S.GATE_OK, S.GATE_OK, S.GATE_DEPTH, S.GATE_DEPTH]
    assert r.z_left[3] < 0
    np.testing.assert_allclose(r.z_left[:3], f * b / np.array([0.875, 1.25, 0.5]), rtol=1e-10)


def test_depth_range():
    f, b = 460.0, 0.11
    rig = S.Rig(kl=(f, f, 375.5, 239.5), kr=(f, f, 375.5, 239.5), R=np.eye(3), t=np.array([-b, 0.0, 0.0]))
    z = np.array([0.3, 0.45, 2.0, 7.9, 8.1])
    d = f * b / z
    pl = np.tile([[400.0, 250.0]], (5, 1))
    pr = pl - np.stack([d, np.zeros(5)], 1)
    r = S.stereo_gate(pl, pr, None, rig, S.GateParams(z_min=0.4, z_max=8.0))
    assert list(r.reason) == [S.GATE_DEPTH, S.GATE_OK, S.GATE_OK, S.GATE_OK, S.GATE_DEPTH]


def test_vertical_misalignment_splits_between_views():
    f, b = 460.0, 0.11
    rig = S.Rig(kl=(f, f, 375.5, 239.5), kr=(f, f, 375.5, 239.5), R=np.eye(3), t=np.array([-b, 0.0, 0.0]))
    e = np.array([0.2, 1.0, 2.0, 2.9, 3.1, 5.0])
    pl = np.tile([[420.0, 260.0]], (len(e), 1))
    pr = pl + np.stack([np.full(len(e), -10.0), e], 1)
    r = S.stereo_gate(pl, pr, None, rig, S.GateParams())
    # equal rows for every 3-D point: the two row errors add up to at least e
    assert (r.e_left + r.e_right >= e * (1 - 1e-9)).all()
    # the linear method splits it almost evenly (symmetric rig)
    np.testing.assert_allclose(r.e_left, e / 2, rtol=0.02)
    np.testing.assert_allclose(r.e_right, e / 2, rtol=0.02)
    assert list(r.reason) == [S.GATE_OK] * 4 + [S.GATE_REPROJ] * 2


def test_untracked_and_non_finite_pairs():
    f = 460.0
    rig = S.Rig(kl=(f, f, 375.5, 239.5), kr=(f, f, 375.5, 239.5), R=np.eye(3), t=np.array([-0.11, 0.0, 0.0]))
    pl = np.array([[300.0, 200.0], [300.0, 200.0], [np.nan, 200.0], [300.0, 200.0]])
    pr = np.array([[290.0, 200.0], [290.0, 200.0], [290.0, 200.0], [290.0, np.inf]])
    r = S.stereo_gate(pl, pr, np.array([1, 0, 1, 1], np.uint8), rig, S.GateParams())
    assert list(r.reason) == [S.GATE_OK, S.GATE_INPUT, S.GATE_INPUT, S.GATE_INPUT]
    assert (r.xyz[1:] == 0).all()


def test_reprojection_uses_both_views():
    """A point seen exactly in the left view but off the epipolar line in the
    right one fails on the right view's error; the left error alone is small."""
    rig, rng = _general_rig(5)
    XL = np.array([[0.3, -0.2, 4.0]])
    pl, pr = _observe(rig.kl, XL), _observe(rig.kr, XL @ rig.R.T + rig.t)
    pr_bad = pr + np.array([[0.0, 6.0]])
    r = S.stereo_gate(np.vstack([pl, pl]), np.vstack([pr, pr_bad]), None, rig, S.GateParams())
    assert list(r.reason) == [S.GATE_OK, S.GATE_REPROJ]
    assert r.e_left[1] + r.e_right[1] > 2.5


def test_each_view_bounds_its_own_error():
    """With a right focal length four times the left one the linear method
    leaves about four times the pixel error in the right view: 0.5 px left,
    2 px right is rejected (each view must be within 1.5 px), although the
    two errors average 1.25 px."""
    rig = S.Rig(kl=(400.0, 400.0, 320.0, 240.0), kr=(1600.0, 1600.0, 320.0, 240.0), R=np.eye(3),
                t=np.array([-0.2, 0.0, 0.0]))
    X = np.array([[0.1, 0.05, 3.0]])
    pl = _observe(rig.kl, X)
    pr = _observe(rig.kr, X + rig.t)
    r0 = S.stereo_gate(pl, pr, None, rig, S.GateParams())
    assert r0.status[0] == 1
    delta = 4.0 / 1600.0  # normalised vertical offset: split evenly, 0.5 px left and 2 px right
    r = S.stereo_gate(pl, pr + np.array([[0.0, 1600.0 * delta]]), None, rig, S.GateParams())
    assert 0.3 < r.e_left[0] < 0.7 and 1.8 < r.e_right[0] < 2.2, (r.e_left, r.e_right)
    assert r.reason[0] == S.GATE_REPROJ


def test_point_behind_the_right_camera_is_rejected():
    """Right camera 1 m ahead of the left one: a point 0.5 m in front of the
    left camera is behind the right one; its projections are still
    consistent (the projective equations ignore the sign), so only the
    right-camera depth test rejects it."""
    rig = S.Rig(kl=(460.0, 460.0, 375.5, 239.5), kr=(460.0, 460.0, 375.5, 239.5), R=np.eye(3),
                t=np.array([-0.1, 0.0, -1.0]))
    X = np.array([[0.2, 0.1, 0.5], [0.2, 0.1, 3.0]])
    pl = _observe(rig.kl, X)
    pr = _observe(rig.kr, X + rig.t)
    r = S.stereo_gate(pl, pr, None, rig, S.GateParams(min_disp=0.5))
    assert list(r.reason) == [S.GATE_DEPTH, S.GATE_OK]
    np.testing.assert_allclose(r.z_left, [0.5, 3.0], rtol=1e-5)
    assert r.z_right[0] < 0
