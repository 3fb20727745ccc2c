"""FP64 oracle of the stereo triangulation gate (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU legs)
may import this module.  It shares no code with the CUDA library.

What it computes (Sec. III-C, Deep Learning Feature Matching): stereo
correspondences are checked against the calibrated rig.  A pair whose
disparity is negligible is dropped; the others are triangulated with the
stereo extrinsics and kept only when the point has a positive depth inside a
valid range and reprojects to within 1.5 px of the observation in both views.
The paper fixes only the 1.5 px; the rest is this reading:

* cameras    pinhole K = (fx, fy, cx, cy) per camera, observations already
             undistorted; X_R = R X_L + t (R row-major, t in metres);
* disparity  |p_R - pi_R(R xbar_L)|, xbar_L = K_L^-1 (p_L, 1): the distance in
             the right image between the observation and the image of the left
             ray's point at infinity (the infinite homography).  When that
             point lies behind the right camera ((R xbar_L)_z <= 0) the
             disparity is taken as infinite.  Kept when disparity > min_disp;
* triangulation  the linear (DLT) two-view method on normalised coordinates
             with P_L = [I | 0], P_R = [R | t]: the homogeneous X is the right
             singular vector of the smallest singular value of the 4x4 matrix
             whose rows are x P^3 - P^1 and y P^3 - P^2 for each view;
* depth      Z_L = X_3 / X_4 and Z_R = (R X + t)_z; kept when X_4 != 0,
             Z_R > 0 and z_min <= Z_L <= z_max;
* reprojection  e_L = |pi_L(X) - p_L|, e_R = |pi_R(R X + t) - p_R| (px); kept
             when max(e_L, e_R) <= max_reproj (1.5 px, inclusive);
* order      an untracked or non-finite pair is rejected first (INPUT), then
             disparity (DISP), depth (DEPTH), reprojection (REPROJ).  ``xyz``
             is the triangulated point (left-camera frame) whenever
             triangulation ran and X_4 != 0, else 0.

Parity note: a status decision is compared only where the oracle's distance
to the threshold it tested last (``margin``, in that test's own unit) is not
tiny; the CUDA path evaluates the same quantities in FP64 by another route
(Jacobi eigen-decomposition of A^T A instead of an SVD of A).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GATE_OK, GATE_INPUT, GATE_DISP, GATE_DEPTH, GATE_REPROJ = 0, 4, 5, 6, 7


@dataclass
class Rig:
    kl: tuple  # fx, fy, cx, cy of the left camera (px)
    kr: tuple  # of the right camera
    R: np.ndarray = field(default_factory=lambda: np.eye(3))  # left -> right rotation
    t: np.ndarray = field(default_factory=lambda: np.zeros(3))  # left -> right translation (m)


@dataclass
class GateParams:
    min_disp: float = 1.0
    z_min: float = 0.1
    z_max: float = 50.0
    max_reproj: float = 1.5


@dataclass
class GateResult:
    xyz: np.ndarray  # [n, 3] float64
    status: np.ndarray  # uint8
    reason: np.ndarray  # uint8
    disparity: np.ndarray  # px (inf where undefined)
    z_left: np.ndarray
    z_right: np.ndarray
    e_left: np.ndarray
    e_right: np.ndarray
    margin: np.ndarray  # distance of the deciding value to its threshold


def _to_norm(K, p):
    fx, fy, cx, cy = (float(v) for v in K)
    return np.stack([(p[:, 0] - cx) / fx, (p[:, 1] - cy) / fy], axis=1)


def _project(K, X):
    fx, fy, cx, cy = (float(v) for v in K)
    return np.stack([fx * X[:, 0] / X[:, 2] + cx, fy * X[:, 1] / X[:, 2] + cy], axis=1)


def triangulate_dlt(xl: np.ndarray, xr: np.ndarray, R: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Homogeneous DLT points [n, 4] from normalised coordinates xl, xr [n, 2]."""
    PL = np.hstack([np.eye(3), np.zeros((3, 1))])
    PR = np.hstack([np.asarray(R, np.float64), np.asarray(t, np.float64).reshape(3, 1)])
    n = xl.shape[0]
    A = np.empty((n, 4, 4))
    A[:, 0] = xl[:, :1] * PL[2] - PL[0]
    A[:, 1] = xl[:, 1:] * PL[2] - PL[1]
    A[:, 2] = xr[:, :1] * PR[2] - PR[0]
    A[:, 3] = xr[:, 1:] * PR[2] - PR[1]
    if n == 0:
        return np.zeros((0, 4))
    _, _, vh = np.linalg.svd(A)
    return vh[:, -1, :]


def stereo_gate(pts_l, pts_r, status_in, rig: Rig, prm: GateParams) -> GateResult:
    pl = np.asarray(pts_l, np.float32).astype(np.float64).reshape(-1, 2)
    pr = np.asarray(pts_r, np.float32).astype(np.float64).reshape(-1, 2)
    n = pl.shape[0]
    st_in = np.ones(n, bool) if status_in is None else np.asarray(status_in).reshape(-1) != 0
    R = np.asarray(rig.R, np.float64).reshape(3, 3)
    t = np.asarray(rig.t, np.float64).reshape(3)

    reason = np.full(n, GATE_OK, np.uint8)
    margin = np.full(n, np.inf)
    finite = np.isfinite(pl).all(axis=1) & np.isfinite(pr).all(axis=1)
    reason[~(st_in & finite)] = GATE_INPUT
    pl = np.where(finite[:, None], pl, 0.0)
    pr = np.where(finite[:, None], pr, 0.0)

    xl = _to_norm(rig.kl, pl)
    xr = _to_norm(rig.kr, pr)
    ray = np.hstack([xl, np.ones((n, 1))]) @ R.T  # R xbar_L
    disp = np.full(n, np.inf)
    front = ray[:, 2] > 0
    if front.any():
        disp[front] = np.hypot(*(pr[front] - _project(rig.kr, ray[front])).T)
    live = reason == GATE_OK
    rej = live & ~(disp > prm.min_disp)
    reason[rej] = GATE_DISP
    margin[live] = np.abs(disp[live] - prm.min_disp)

    Xh = triangulate_dlt(xl, xr, R, t)
    ok_w = Xh[:, 3] != 0
    X = np.zeros((n, 3))
    X[ok_w] = Xh[ok_w, :3] / Xh[ok_w, 3:]
    XR = X @ R.T + t
    zl, zr = X[:, 2], XR[:, 2]
    live = reason == GATE_OK
    good_z = ok_w & (zr > 0) & (zl >= prm.z_min) & (zl <= prm.z_max)
    reason[live & ~good_z] = GATE_DEPTH
    mz = np.minimum(np.minimum(np.abs(zl - prm.z_min), np.abs(zl - prm.z_max)), np.abs(zr))
    margin[live] = np.minimum(margin[live], mz[live])

    el = np.full(n, np.inf)
    er = np.full(n, np.inf)
    live = reason == GATE_OK
    if live.any():
        el[live] = np.hypot(*(_project(rig.kl, X[live]) - pl[live]).T)
        er[live] = np.hypot(*(_project(rig.kr, XR[live]) - pr[live]).T)
    emax = np.maximum(el, er)
    reason[live & ~(emax <= prm.max_reproj)] = GATE_REPROJ
    margin[live] = np.minimum(margin[live], np.abs(emax[live] - prm.max_reproj))

    tri = (reason == GATE_OK) | (reason == GATE_DEPTH) | (reason == GATE_REPROJ)
    xyz = np.where((tri & ok_w)[:, None], X, 0.0)
    return GateResult(xyz, (reason == GATE_OK).astype(np.uint8), reason, disp, zl, zr, el, er, margin)
