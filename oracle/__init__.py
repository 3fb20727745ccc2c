"""FP64 CPU oracle for the pyramidal Lucas-Kanade hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and its reference arm) may import this package.  It shares no code with
the CUDA library.  The arithmetic lives in ``orc.c``; this module only
marshals numpy arrays.  Readings of the paper it implements are listed at the
top of ``orc.c``; Sec. IV (Shi-Tomasi + LK optical flow), Sec. III-A (LK needs
keypoints only) and Sec. V-A (cross-camera optical-flow verification) are the
passages it follows.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

LOST_EIG, LOST_OOB, LOST_FB, LOST_INPUT = 1, 2, 3, 4

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_oracle())
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        i16p = np.ctypeslib.ndpointer(np.int16, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        lib.orc_pyrdown.argtypes = [u8p, C.c_int, C.c_int, C.c_int, u8p, C.c_int]
        lib.orc_scharr.argtypes = [u8p, C.c_int, C.c_int, C.c_int, i16p, i16p, C.c_int]
        lib.orc_track.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, f64p, C.c_void_p, C.c_int,
                                  f64p, u8p, f64p, u8p, i32p, f64p, f64p, C.c_void_p]
        lib.orc_fb_check.argtypes = [f64p, f64p, u8p, u8p, C.c_int, C.c_double, u8p, f64p, f64p]
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
        lib.orc_gftt.restype = C.c_int
        lib.orc_gftt.argtypes = [i16p, i16p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_int, C.c_int,
                                 C.c_int, C.c_void_p, C.c_int, C.c_int, i32p, f32p]
        lib.orc_gftt_score.restype = C.c_float
        lib.orc_gftt_score.argtypes = [C.c_long, C.c_long, C.c_long]
        _lib = lib
    return _lib


class _Level(C.Structure):
    _fields_ = [("img", C.c_void_p), ("gx", C.c_void_p), ("gy", C.c_void_p), ("w", C.c_int), ("h", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("win", C.c_int), ("levels", C.c_int), ("max_iters", C.c_int), ("eps", C.c_double),
                ("min_eig", C.c_double)]


# ------------------------------------------------------------------ pyramid
def pyr_down(src: np.ndarray) -> np.ndarray:
    src = np.ascontiguousarray(src, dtype=np.uint8)
    h, w = src.shape
    dst = np.zeros(((h + 1) // 2, (w + 1) // 2), dtype=np.uint8)
    _load().orc_pyrdown(src, w, h, w, dst, dst.shape[1])
    return dst


def pyramid(img: np.ndarray, levels: int) -> list:
    """Levels 0..levels-1; level 0 is a copy of ``img``."""
    out = [np.ascontiguousarray(img, dtype=np.uint8).copy()]
    for _ in range(1, levels):
        out.append(pyr_down(out[-1]))
    return out


def scharr(img: np.ndarray):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    gx = np.zeros((h, w), dtype=np.int16)
    gy = np.zeros((h, w), dtype=np.int16)
    _load().orc_scharr(img, w, h, w, gx, gy, w)
    return gx, gy


@dataclass
class Pyramid:
    levels: list  # uint8 images
    gx: list  # int16 raw Scharr
    gy: list


def build_pyramid(img: np.ndarray, levels: int) -> Pyramid:
    lv = pyramid(img, levels)
    g = [scharr(a) for a in lv]
    return Pyramid(lv, [a for a, _ in g], [b for _, b in g])


# ------------------------------------------------------------------ tracking
@dataclass
class TrackResult:
    pts: np.ndarray  # float64 [n, 2]
    status: np.ndarray  # uint8 [n]
    err: np.ndarray  # float64 [n]
    reason: np.ndarray  # uint8 [n]
    iters: np.ndarray  # int32 [n]
    lmin: np.ndarray  # float64 [n]
    margin: np.ndarray  # float64 [n, 4]: eig (relative), conv at every iteration (px), bound (px),
    #                     conv at the iterations that stopped a level (px)
    iters_level: np.ndarray | None = None  # int32 [n, levels]: Newton iterations per level (on request)

    def decision_margin(self, reason: int) -> np.ndarray:
        """Per point, the smallest margin of the status decisions of one kind
        (a LOST_* code): the eigenvalue test (relative) or the image-bound test
        (px); other kinds are not decided by a single pass (infinite)."""
        if reason == LOST_EIG:
            return self.margin[:, 0]
        if reason == LOST_OOB:
            return self.margin[:, 2]
        return np.full(self.margin.shape[0], np.inf)


def _levels_struct(levels_f64):
    """levels_f64: list of (img, gx, gy) float64 arrays (gx, gy may be None)."""
    keep = []
    arr = (_Level * len(levels_f64))()
    for k, (img, gx, gy) in enumerate(levels_f64):
        img = np.ascontiguousarray(img, dtype=np.float64)
        keep.append(img)
        arr[k].img = img.ctypes.data
        if gx is not None:
            gx = np.ascontiguousarray(gx, dtype=np.float64)
            gy = np.ascontiguousarray(gy, dtype=np.float64)
            keep += [gx, gy]
            arr[k].gx, arr[k].gy = gx.ctypes.data, gy.ctypes.data
        arr[k].h, arr[k].w = img.shape
    return arr, keep


def track_f64(levels_I, levels_J, pts, win=21, levels=None, max_iters=30, eps=0.01, min_eig=1e-4,
              guess=None, per_level=False) -> TrackResult:
    """Core LK on double-valued levels.  ``levels_I``: list of (img, gx, gy)
    with gradients in grey levels per pixel; ``levels_J``: list of images."""
    L = len(levels_I) if levels is None else levels
    if win % 2 != 1 or win < 3:
        raise ValueError("window side must be odd and >= 3")
    if L < 1 or L > len(levels_I) or L > len(levels_J):
        raise ValueError("levels out of range")
    Is, k1 = _levels_struct(levels_I)
    Js, k2 = _levels_struct([(j, None, None) for j in levels_J])
    prm = _Params(win, L, max_iters, eps, min_eig)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    n = pts.shape[0]
    g = None
    if guess is not None:
        g = np.ascontiguousarray(guess, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((n, 2))
    st = np.zeros(n, np.uint8)
    err = np.zeros(n)
    rs = np.zeros(n, np.uint8)
    it = np.zeros(n, np.int32)
    lm = np.zeros(n)
    mg = np.zeros((n, 4))
    il = np.zeros((n, L), np.int32) if per_level else None
    _load().orc_track(C.addressof(Is), C.addressof(Js), C.addressof(prm), pts,
                      None if g is None else g.ctypes.data, n, out, st, err, rs, it, lm, mg,
                      None if il is None else il.ctypes.data)
    return TrackResult(out, st, err, rs, it, lm, mg, il)


def track(pI: Pyramid, pJ: Pyramid, pts, win=21, levels=None, max_iters=30, eps=0.01, min_eig=1e-4,
          guess=None, per_level=False) -> TrackResult:
    """LK from pyramid ``pI`` to ``pJ`` on uint8 levels and raw int16 Scharr
    gradients (converted to grey levels per pixel by the factor 1/32)."""
    L = len(pI.levels) if levels is None else levels
    lvI = [(pI.levels[k].astype(np.float64), pI.gx[k] / 32.0, pI.gy[k] / 32.0) for k in range(L)]
    lvJ = [pJ.levels[k].astype(np.float64) for k in range(L)]
    return track_f64(lvI, lvJ, pts, win, L, max_iters, eps, min_eig, guess, per_level)


def fb_check(p0, p0_back, st_f, st_b, thr=0.5):
    p0 = np.ascontiguousarray(p0, dtype=np.float64).reshape(-1, 2)
    p1 = np.ascontiguousarray(p0_back, dtype=np.float64).reshape(-1, 2)
    n = p0.shape[0]
    st = np.zeros(n, np.uint8)
    d = np.zeros(n)
    m = np.zeros(n)
    _load().orc_fb_check(p0, p1, np.ascontiguousarray(st_f, np.uint8), np.ascontiguousarray(st_b, np.uint8),
                         n, float(thr), st, d, m)
    return st, d, m


@dataclass
class FBResult:
    fwd: TrackResult
    bwd: TrackResult
    status: np.ndarray  # forward-backward checked status
    reason: np.ndarray
    fb_dist: np.ndarray
    fb_margin: np.ndarray

    def min_margin(self) -> np.ndarray:
        """Smallest threshold margin over both passes and the FB test
        (eigenvalue margins are relative, the others in pixels)."""
        return np.minimum(np.minimum(self.fwd.margin.min(axis=1), self.bwd.margin.min(axis=1)),
                          self.fb_margin)

    def decision_margin(self, reason: int) -> np.ndarray:
        """Per point, the smallest margin of the status decisions of one kind
        (a LOST_* code) over both passes; LOST_INPUT decisions are exact."""
        if reason == LOST_FB:
            return self.fb_margin
        return np.minimum(self.fwd.decision_margin(reason), self.bwd.decision_margin(reason))


def track_fb(pI: Pyramid, pJ: Pyramid, pts, win=21, levels=None, max_iters=30, eps=0.01, min_eig=1e-4,
             fb_thr=0.5, per_level=False) -> FBResult:
    """Forward I->J from ``pts``, backward J->I from the forward result, FB test.

    The stereo gate of Sec. V-A (only features passing the cross-camera
    optical-flow check enter the pool) is this call with (I, J) = (left, right)."""
    f = track(pI, pJ, pts, win, levels, max_iters, eps, min_eig, per_level=per_level)
    b = track(pJ, pI, f.pts, win, levels, max_iters, eps, min_eig, per_level=per_level)
    st, d, m = fb_check(pts, b.pts, f.status, b.status, fb_thr)
    reason = f.reason.copy()
    reason[(reason == 0)] = b.reason[(reason == 0)]
    reason[(reason == 0) & (st == 0)] = LOST_FB
    return FBResult(f, b, st, reason, d, m)


def gftt(gx, gy, max_corners=150, quality=0.01, min_dist=10, nms_radius=4, block_radius=1, border=10, mask=None):
    """Shi-Tomasi corners of one level from its raw int16 Scharr planes (the
    reading is stated in orc.c).  Returns (corners int32 [k, 2], scores
    float32 [k]) in priority order."""
    gx = np.ascontiguousarray(gx, np.int16)
    gy = np.ascontiguousarray(gy, np.int16)
    h, w = gx.shape
    m = None if mask is None else np.ascontiguousarray(mask, np.float64).reshape(-1, 2)
    out = np.zeros((max(1, max_corners), 2), np.int32)
    sc = np.zeros(max(1, max_corners), np.float32)
    k = _load().orc_gftt(gx, gy, w, h, w, block_radius, quality, nms_radius, border, min_dist,
                         None if m is None else m.ctypes.data, 0 if m is None else len(m), max_corners, out, sc)
    return out[:k].copy(), sc[:k].copy()


def gftt_score(a, b, c):
    """Single-precision minimum eigenvalue of [[a, b], [b, c]] as the detector evaluates it."""
    return float(_load().orc_gftt_score(int(a), int(b), int(c)))
