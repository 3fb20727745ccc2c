"""Workload builders: frame pairs, stereo sequences and camera-stream mixes.

* ``make_config1``: one 752x480 mono pair.  Frame 2 is the continuous texture
  seen through a 1 degree rotation about the image centre plus a seeded
  sub-pixel translation |t| <= 8 px, evaluated exactly (no resampling); the
  ground-truth position of every keypoint is known in closed form.
* ``HeightFieldScene`` / ``make_stereo_sequence``: a textured wall whose depth
  is a tilted plane at 2-5 m plus seeded Gaussian bumps, seen by a calibrated
  stereo pair (baseline 0.11 m, f = 460 px at 752x480) moving at <= 0.3 m/s
  (20 Hz) and rotating <= 5 degrees per frame.  Rays are cast per pixel on the
  CPU (fixed-point iteration on the depth field); the texture is a raster
  sampled with cubic B-spline interpolation.  The optional motion blur and
  exposure change give the 1280x1024 precision-variant workload.
* ``make_stream_mix`` / ``render_stream_frames``: independent camera streams of
  uneven shapes (640x480, 752x480, 960x600, 1440x1080, 1920x1200), mono or
  stereo, 200-2000 keypoints and 4-6 pyramid levels each, with frames related
  by small rigid motions of an exactly evaluated texture.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage

from .keypoints import select_keypoints_nms, select_keypoints_topfrac
from .texture import BlobTexture, affine_from_motion, invert_affine, quantize_u8

IDENTITY = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


# --------------------------------------------------------------------- config 1
@dataclass
class Config1Pair:
    I: np.ndarray  # uint8 [h, w], previous frame
    J: np.ndarray  # uint8 [h, w], current frame
    pts: np.ndarray  # float32 [n, 2] keypoints in I
    gt: np.ndarray  # float64 [n, 2] exact positions of the keypoints in J
    motion: np.ndarray  # 2x3 rigid motion I -> J
    seed: int
    params: dict = field(default_factory=dict)


def make_config1(seed: int = 1, w: int = 752, h: int = 480, n: int = 150, theta_deg: float = 1.0,
                 max_shift: float = 8.0, margin: float = 28.0) -> Config1Pair:
    rng = np.random.Generator(np.random.PCG64(seed))
    tex = BlobTexture(seed * 7919 + 1, extent=(-60.0, -60.0, w + 60.0, h + 60.0))
    I = quantize_u8(tex.eval_affine(w, h, IDENTITY))
    # |t| <= max_shift: radius and angle drawn separately (sub-pixel by construction)
    r = rng.uniform(0.25 * max_shift, max_shift)
    a = rng.uniform(0.0, 2.0 * np.pi)
    tx, ty = r * np.cos(a), r * np.sin(a)
    M = affine_from_motion(theta_deg, tx, ty, (w - 1) / 2.0, (h - 1) / 2.0)
    J = quantize_u8(tex.eval_affine(w, h, invert_affine(M)))
    pts = select_keypoints_topfrac(I, n, seed * 7919 + 2, margin=margin)
    p = pts.astype(np.float64)
    gt = p @ M[:, :2].T + M[:, 2]
    return Config1Pair(I=I, J=J, pts=pts, gt=gt, motion=M, seed=seed,
                       params=dict(win=21, levels=4, max_iters=30, eps=0.01, fb_thr=0.5, min_eig=1e-4))


# ---------------------------------------------------------------- height field
def _rot(yaw: float, pitch: float, roll: float) -> np.ndarray:
    cy, sy = np.cos(yaw), np.sin(yaw)
    cp, sp = np.cos(pitch), np.sin(pitch)
    cr, sr = np.cos(roll), np.sin(roll)
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    Rz = np.array([[cr, -sr, 0], [sr, cr, 0], [0, 0, 1]])
    return Ry @ Rx @ Rz


class HeightFieldScene:
    """Textured wall Z = D(X, Y) in front of a moving stereo camera.

    World axes follow the camera convention (X right, Y down, Z forward)."""

    TEXEL_M = 0.0087  # one texture pixel, about one image pixel at 4 m and f = 460
    OVERSAMPLE = 2  # raster cells per texture pixel
    EXTENT = (-8.0, -6.0, 8.0, 6.0)  # metres

    def __init__(self, seed: int, n_bumps: int = 40, texel_m: float | None = None):
        """texel_m: size of one texture pixel on the wall; a camera with a
        larger focal length should get a proportionally smaller texel so that
        the texture keeps its detail per image pixel."""
        if texel_m is not None:
            self.TEXEL_M = float(texel_m)
        rng = np.random.Generator(np.random.PCG64(seed))
        x0, y0, x1, y1 = self.EXTENT
        self.z0 = rng.uniform(3.0, 4.0)
        self.sx = rng.uniform(-0.12, 0.12)
        self.sy = rng.uniform(-0.12, 0.12)
        # bumps: separable Gaussians, rastered at 2 cm and sampled with cubic splines
        bx = rng.uniform(x0, x1, n_bumps)
        by = rng.uniform(y0, y1, n_bumps)
        bs = rng.uniform(0.2, 0.8, n_bumps)
        ba = rng.uniform(-0.35, 0.35, n_bumps)
        self.bump_res = 0.02
        gxs = np.arange(x0, x1 + 1e-9, self.bump_res)
        gys = np.arange(y0, y1 + 1e-9, self.bump_res)
        Gx = np.exp(-((gxs[:, None] - bx) ** 2) / (2 * bs**2))
        Gy = np.exp(-((gys[:, None] - by) ** 2) / (2 * bs**2))
        bumps = (Gy * ba) @ Gx.T
        self.bump_coef = ndimage.spline_filter(bumps, order=3, mode="nearest")
        # wall texture in texture pixels; blob density matches 400 per 752x480
        tw = (x1 - x0) / self.TEXEL_M
        th = (y1 - y0) / self.TEXEL_M
        n_blobs = int(round(400 * tw * th / (752 * 480)))
        tex = BlobTexture(seed * 104729 + 3, extent=(0.0, 0.0, tw, th), n_blobs=n_blobs)
        k = self.OVERSAMPLE
        rw, rh = int(np.ceil(tw * k)), int(np.ceil(th * k))
        raster = tex.eval_affine(rw, rh, np.array([[1.0 / k, 0, 0], [0, 1.0 / k, 0]]))
        self.tex_coef = ndimage.spline_filter(raster, order=3, mode="nearest")
        self.base = tex.base

    def depth(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        x0, y0, _, _ = self.EXTENT
        bi = ndimage.map_coordinates(
            self.bump_coef, [(Y - y0) / self.bump_res, (X - x0) / self.bump_res],
            order=3, mode="nearest", prefilter=False)
        return self.z0 + self.sx * X + self.sy * Y + bi

    def render(self, R: np.ndarray, C: np.ndarray, w: int, h: int, f: float, iters: int = 10):
        """Float image [h, w] and depth map seen by a pinhole camera (R, C)."""
        cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
        xs = (np.arange(w) - cx) / f
        ys = (np.arange(h) - cy) / f
        dc = np.stack(np.broadcast_arrays(xs[None, :], ys[:, None], np.ones((h, w))), axis=-1)
        d = dc @ R.T
        dx, dy, dz = d[..., 0], d[..., 1], d[..., 2]
        t = (self.z0 - C[2]) / dz
        for _ in range(iters):
            X = C[0] + t * dx
            Y = C[1] + t * dy
            t = (self.depth(X, Y) - C[2]) / dz
        X = C[0] + t * dx
        Y = C[1] + t * dy
        x0, y0, _, _ = self.EXTENT
        k = self.OVERSAMPLE / self.TEXEL_M
        img = ndimage.map_coordinates(self.tex_coef, [(Y - y0) * k, (X - x0) * k], order=3,
                                      mode="constant", cval=self.base, prefilter=False)
        return img, t * dz


def _motion_blur(img: np.ndarray, length: float, angle: float) -> np.ndarray:
    if length < 1.0:
        return img
    n = 64
    s = np.linspace(-0.5, 0.5, n) * length
    xs = np.rint(s * np.cos(angle)).astype(int)
    ys = np.rint(s * np.sin(angle)).astype(int)
    r = int(np.ceil(length / 2.0)) + 1
    k = np.zeros((2 * r + 1, 2 * r + 1))
    np.add.at(k, (ys + r, xs + r), 1.0)
    k /= k.sum()
    return ndimage.convolve(img, k, mode="nearest")


@dataclass
class StereoSequence:
    left: list  # uint8 [h, w] per frame
    right: list
    depth: list  # float32 depth of the left camera per frame
    kps: list  # float32 [n, 2] per frame, on the left image
    poses: list  # (R, C) of the left camera
    f: float
    baseline: float
    seed: int
    gains: list


def _render_stereo_frame(args):
    """One frame of a stereo sequence (left, right, left depth, keypoints)."""
    scene, R, C, CR, w, h, f, blur, g, kp_seed, n_kp, nms_radius = args
    imL, dL = scene.render(R, C, w, h, f)
    imR, _ = scene.render(R, CR, w, h, f)
    if blur is not None:
        imL = _motion_blur(imL, *blur)
        imR = _motion_blur(imR, *blur)
    L8 = quantize_u8((imL - 128.0) * g + 128.0 if g != 1.0 else imL)
    R8 = quantize_u8((imR - 128.0) * g + 128.0 if g != 1.0 else imR)
    return L8, R8, dL.astype(np.float32), select_keypoints_nms(L8, n_kp, kp_seed, radius=nms_radius)


def make_stereo_sequence(seed: int = 2, n_frames: int = 4, w: int = 752, h: int = 480, n_kp: int = 1000,
                         f: float | None = None, baseline: float = 0.11, fps: float = 20.0,
                         max_speed: float = 0.3, max_rot_deg: float = 5.0, blur_max: float = 0.0,
                         gain_range: tuple[float, float] | None = None, nms_radius: int = 4,
                         scene: HeightFieldScene | None = None, map_fn=map) -> StereoSequence:
    """``map_fn``: how the frames are rendered (e.g. a process pool's map);
    the frames do not depend on it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if f is None:
        f = 460.0 * w / 752.0
    scene = scene or HeightFieldScene(seed, texel_m=HeightFieldScene.TEXEL_M * 460.0 / f)
    # smooth trajectory: per-axis sinusoids, peak speed <= max_speed and
    # peak rotation rate <= max_rot_deg per frame (split over three axes)
    per_axis_v = max_speed / fps / np.sqrt(3.0)
    per_axis_w = np.deg2rad(max_rot_deg) / np.sqrt(3.0)
    Pt = rng.uniform(40.0, 120.0, 3)
    vt = rng.uniform(0.3, 1.0, 3) * per_axis_v
    pht = rng.uniform(0, 2 * np.pi, 3)
    Pr = rng.uniform(30.0, 90.0, 3)
    wr = rng.uniform(0.3, 1.0, 3) * per_axis_w
    phr = rng.uniform(0, 2 * np.pi, 3)
    jobs, poses, gains = [], [], []
    for k in range(n_frames):
        C = vt * Pt / (2 * np.pi) * np.sin(2 * np.pi * k / Pt + pht)
        ang = wr * Pr / (2 * np.pi) * np.sin(2 * np.pi * k / Pr + phr)
        R = _rot(*ang)
        CR = C + R @ np.array([baseline, 0.0, 0.0])
        blur = None
        if blur_max > 0:
            bl, ba = rng.uniform(0, blur_max), rng.uniform(0, np.pi)
            blur = (bl, ba)
        g = 1.0
        if gain_range is not None and k > 0:
            g = rng.uniform(*gain_range)
        jobs.append((scene, R, C, CR, w, h, f, blur, g, seed * 31 + k, n_kp, nms_radius))
        poses.append((R, C))
        gains.append(g)
    out = list(map_fn(_render_stereo_frame, jobs))
    return StereoSequence([o[0] for o in out], [o[1] for o in out], [o[2] for o in out], [o[3] for o in out],
                          poses, f, baseline, seed, gains)


def make_config3_pair(seed: int = 3, n_frames: int = 2, w: int = 1280, h: int = 1024, n_kp: int = 2000):
    """1280x1024 stereo sequence with motion blur (0-7 px) and exposure gain
    U[0.7, 1.3] on every frame after the first."""
    return make_stereo_sequence(seed=seed, n_frames=n_frames, w=w, h=h, n_kp=n_kp,
                                blur_max=7.0, gain_range=(0.7, 1.3))


def _render_polygons(w, h, polys, base=128.0, ss=4):
    """Area-sampled rendering of filled convex polygons (painter's order) on
    a constant background: each pixel is the mean of an ss x ss grid of
    sub-samples, so edges are sharp (one pixel of transition) and exact."""
    img = np.full((h, w), base, np.float64)
    off = (np.arange(ss) + 0.5) / ss - 0.5
    for verts, val in polys:
        x0 = max(0, int(np.floor(verts[:, 0].min())) - 1)
        x1 = min(w, int(np.ceil(verts[:, 0].max())) + 2)
        y0 = max(0, int(np.floor(verts[:, 1].min())) - 1)
        y1 = min(h, int(np.ceil(verts[:, 1].max())) + 2)
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        sx = np.broadcast_to(xx[:, :, None, None] + off[None, None, None, :], xx.shape + (ss, ss))
        sy = np.broadcast_to(yy[:, :, None, None] + off[None, None, :, None], xx.shape + (ss, ss))
        inside = np.ones(sx.shape, bool)
        n = len(verts)
        area = 0.0
        for k in range(n):
            (ax, ay), (bx, by) = verts[k], verts[(k + 1) % n]
            area += ax * by - bx * ay
        sgn = 1.0 if area > 0 else -1.0
        for k in range(n):
            (ax, ay), (bx, by) = verts[k], verts[(k + 1) % n]
            inside &= sgn * ((bx - ax) * (sy - ay) - (by - ay) * (sx - ax)) >= 0
        cov = inside.mean(axis=(2, 3))
        img[y0:y1, x0:x1] = img[y0:y1, x0:x1] * (1 - cov) + val * cov
    return img


@dataclass
class ContrastPair:
    I: np.ndarray
    J: np.ndarray
    pts: np.ndarray  # float32 [n, 2] keypoints in I
    gt: np.ndarray  # float64 [n, 2] positions of the keypoints under the scene motion
    gain: float
    seed: int


def make_config3_contrast_pair(seed: int = 5, w: int = 1280, h: int = 1024, n_kp: int = 2000,
                               n_rects: int = 900, gain: float = 1.3) -> ContrastPair:
    """High-contrast variant of the precision workload: unblurred step edges
    (rotated rectangles of grey levels 16-240 on a mid-grey background,
    area-sampled), the second frame the same scene under a small rigid motion
    (rotation up to 0.5 degrees, translation up to 5 px, sub-pixel) with
    exposure x `gain` about mid-grey.  Step edges of contrast above 128 give
    Scharr responses above 2048, where half-precision storage of raw/32
    rounds the odd ones."""
    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for _ in range(n_rects):
        cx, cy = rng.uniform(-20, w + 20), rng.uniform(-20, h + 20)
        a, b = rng.uniform(8, 40), rng.uniform(8, 40)
        th = rng.uniform(0, np.pi)
        c, s_ = np.cos(th), np.sin(th)
        corners = np.array([[-a, -b], [a, -b], [a, b], [-a, b]]) @ np.array([[c, s_], [-s_, c]])
        polys.append((corners + [cx, cy], float(rng.choice([rng.uniform(16, 70), rng.uniform(186, 240)]))))
    theta = rng.uniform(-0.5, 0.5)
    r, ang = rng.uniform(1.0, 5.0), rng.uniform(0, 2 * np.pi)
    M = affine_from_motion(theta, r * np.cos(ang), r * np.sin(ang), (w - 1) / 2.0, (h - 1) / 2.0)
    I = quantize_u8(_render_polygons(w, h, polys))
    moved = [(v @ M[:, :2].T + M[:, 2], val) for v, val in polys]
    J = quantize_u8((_render_polygons(w, h, moved) - 128.0) * gain + 128.0)
    pts = select_keypoints_nms(I, n_kp, seed * 31 + 1, radius=4, margin=30.0)
    gt = pts.astype(np.float64) @ M[:, :2].T + M[:, 2]
    return ContrastPair(I, J, pts, gt, gain, seed)


# ----------------------------------------------------------------- stream mix
STREAM_SHAPES = [(640, 480), (752, 480), (960, 600), (1440, 1080), (1920, 1200)]


@dataclass
class StreamSpec:
    sid: int
    w: int
    h: int
    stereo: bool
    n_kp: int
    levels: int
    seed: int


def make_stream_mix(n_streams: int, seed: int = 4, kp_range=(200, 2000), levels=(4, 5, 6)) -> list:
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(n_streams):
        w, h = STREAM_SHAPES[int(rng.integers(0, len(STREAM_SHAPES)))]
        out.append(StreamSpec(sid=s, w=w, h=h, stereo=bool(rng.integers(0, 2)),
                              n_kp=int(rng.integers(kp_range[0], kp_range[1] + 1)),
                              levels=int(levels[int(rng.integers(0, len(levels)))]),
                              seed=seed * 1009 + s))
    return out


@dataclass
class StreamFrames:
    spec: StreamSpec
    left: list
    right: list  # None entries for mono streams
    kps: list  # keypoints on each left frame


def stream_rig(spec: StreamSpec, baseline: float = 0.11):
    """Calibration of a stream's (rectified) stereo rig as plain numbers:
    pinhole (f, f, cx, cy) for both cameras with f = 460 px scaled by the
    width from 752 px and the principal point at the image centre, identity
    rotation and the right camera `baseline` metres along +x (X_R = X_L + t,
    t = (-baseline, 0, 0)).  The constant disparity d of render_stream_frames
    is then a fronto-parallel plane at depth f * baseline / d."""
    f = 460.0 * spec.w / 752.0
    k = (f, f, (spec.w - 1) / 2.0, (spec.h - 1) / 2.0)
    return k, k, (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0), (-baseline, 0.0, 0.0)


def render_stream_frames(spec: StreamSpec, n_frames: int = 4, max_shift: float = 6.0,
                         max_rot_deg: float = 0.5) -> StreamFrames:
    """Frames k = 0..n_frames-1 of one stream: texture under a random walk of
    small rigid motions; the right camera of a stereo stream sees the same
    texture shifted left by a constant seeded disparity (a fronto-parallel
    plane) plus a small vertical misalignment below 0.5 px."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    w, h = spec.w, spec.h
    tex = BlobTexture(spec.seed * 7 + 11, extent=(-120.0, -120.0, w + 120.0, h + 120.0),
                      n_blobs=int(round(400 * (w + 240) * (h + 240) / (752 * 480))), blob_radius_sigmas=4.0)
    disp = rng.uniform(4.0, 24.0)
    vmis = rng.uniform(-0.4, 0.4)
    theta, tx, ty = 0.0, 0.0, 0.0
    left, right, kps = [], [], []
    for k in range(n_frames):
        M = affine_from_motion(theta, tx, ty, (w - 1) / 2.0, (h - 1) / 2.0)
        A = invert_affine(M)
        L = quantize_u8(tex.eval_affine(w, h, A))
        left.append(L)
        if spec.stereo:
            MR = np.array([[1.0, 0.0, -disp], [0.0, 1.0, vmis]])
            AR = invert_affine(np.vstack([MR, [0, 0, 1]])[:2] @ np.vstack([M, [0, 0, 1]]))
            right.append(quantize_u8(tex.eval_affine(w, h, AR)))
        else:
            right.append(None)
        kps.append(select_keypoints_topfrac(L, spec.n_kp, spec.seed * 13 + k, margin=30.0, top_frac=0.3))
        r = rng.uniform(0.3, 1.0) * max_shift
        a = rng.uniform(0, 2 * np.pi)
        tx += r * np.cos(a)
        ty += r * np.sin(a)
        theta += rng.uniform(-max_rot_deg, max_rot_deg)
    return StreamFrames(spec, left, right, kps)
