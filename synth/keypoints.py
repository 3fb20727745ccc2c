"""Seeded keypoint draws on textured pixels.

The score used to pick "textured" pixels is the smaller eigenvalue of a 7x7
box-summed structure tensor of central differences of the rendered image.  It
is a generator heuristic only: the tracking method's own eigenvalue test (on
bilinearly sampled Scharr gradients over the tracking window) lives in the
oracle and in the CUDA library, not here.
"""

from __future__ import annotations

import numpy as np
from scipy import ndimage


def _score(img: np.ndarray) -> np.ndarray:
    f = img.astype(np.float64)
    dy, dx = np.gradient(f)
    sxx = ndimage.uniform_filter(dx * dx, size=7, mode="nearest")
    syy = ndimage.uniform_filter(dy * dy, size=7, mode="nearest")
    sxy = ndimage.uniform_filter(dx * dy, size=7, mode="nearest")
    tr = 0.5 * (sxx + syy)
    return tr - np.sqrt(np.maximum(0.25 * (sxx - syy) ** 2 + sxy * sxy, 0.0))


def _margin_mask(h: int, w: int, margin: float) -> np.ndarray:
    m = int(np.ceil(margin))
    mask = np.zeros((h, w), dtype=bool)
    if h > 2 * m and w > 2 * m:
        mask[m : h - m, m : w - m] = True
    return mask


def select_keypoints_topfrac(
    img: np.ndarray, n: int, seed: int, margin: float = 20.0, top_frac: float = 0.2, jitter: bool = True
) -> np.ndarray:
    """Seeded draw of ``n`` pixels whose score is in the top ``top_frac``.

    Returns float32 [n, 2] (x, y) in level-0 pixels; with ``jitter`` a seeded
    sub-pixel offset U[-0.5, 0.5) is added to each coordinate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h, w = img.shape
    s = _score(img)
    mask = _margin_mask(h, w, margin + 0.5)
    vals = s[mask]
    thr = np.quantile(vals, 1.0 - top_frac)
    ys, xs = np.nonzero(mask & (s >= thr))
    pick = rng.choice(len(xs), size=min(n, len(xs)), replace=False)
    pts = np.stack([xs[pick], ys[pick]], axis=1).astype(np.float64)
    if jitter:
        pts += rng.uniform(-0.5, 0.5, size=pts.shape)
    return pts.astype(np.float32)


def select_keypoints_nms(
    img: np.ndarray, n: int, seed: int, radius: int = 4, margin: float = 20.0, jitter: bool = True
) -> np.ndarray:
    """Learned-extractor-like density: local maxima of the score within a
    (2 radius + 1)^2 neighbourhood, strongest first, seeded sub-pixel jitter.

    If fewer than ``n`` maxima exist, the rest are a seeded draw of other
    in-margin pixels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h, w = img.shape
    s = _score(img)
    mask = _margin_mask(h, w, margin + 0.5)
    mx = ndimage.maximum_filter(s, size=2 * radius + 1, mode="nearest")
    cand = mask & (s >= mx) & (s > 0)
    ys, xs = np.nonzero(cand)
    order = np.argsort(-s[ys, xs], kind="stable")
    ys, xs = ys[order][:n], xs[order][:n]
    pts = np.stack([xs, ys], axis=1).astype(np.float64)
    if len(pts) < n:
        ys2, xs2 = np.nonzero(mask & ~cand)
        extra = rng.choice(len(xs2), size=n - len(pts), replace=False)
        pts = np.concatenate([pts, np.stack([xs2[extra], ys2[extra]], axis=1).astype(np.float64)])
    if jitter:
        pts += rng.uniform(-0.5, 0.5, size=pts.shape)
    return pts.astype(np.float32)
