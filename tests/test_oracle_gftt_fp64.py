"""The detector oracle's single-precision score pinned to the mathematics
(no GPU).

Shi-Tomasi's score is the smaller eigenvalue of the 2x2 structure tensor
[[a, b], [b, c]] (Sec. IV names the detector; the paper gives no precision).
The oracle evaluates lambda = ((a + c) - sqrt((a - c)^2 + 4 b^2)) / 2 in FP32,
operation by operation, so that the kernel can take every decision the same
way.  These tests show that this FP32 evaluation is the exact eigenvalue up
to the rounding of that operation sequence, and that on a realistic image the
corners it selects are the corners an exact (FP64) score selects.

Error bound of the FP32 sequence (u = 2^-24, a, c >= 0, b^2 <= a c):
  fa, fb, fc round a, b, c (relative u each); d = fl(fa - fc) is off from
  a - c by at most 2u (a + c); fl(fb) by u |b| <= u (a + c) / 2.  As
  sqrt(x^2 + y^2) is 1-Lipschitz in (x, y), sqrt(d^2 + 4 fb^2) is off from
  r = sqrt((a - c)^2 + 4 b^2) by at most 3u (a + c); rounding d^2, 4 b^2
  (exact), their sum and the square root adds 1.5u r + u r <= 2.5u (a + c).
  s = fl(fa + fc) is off by at most 2u (a + c), and t = fl(s - r) adds
  u (s - r) <= u (a + c).  So |t - 2 lambda| <= 8.5u (a + c) and
  |score - lambda| <= 4.25u (a + c) (to first order in u; clamping at 0 only
  brings a negative rounding result closer to lambda >= 0).
"""

from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import synth

U = 2.0 ** -24
BOUND = 4.25 * U * (1 + 2.0 ** -20)  # first-order bound, with room for the O(u^2) terms


def _exact_lmin(a: int, b: int, c: int) -> float:
    getcontext().prec = 60
    d = Decimal((a - c) * (a - c) + 4 * b * b).sqrt()
    return float((Decimal(a + c) - d) / 2)


def _tensor(gx, gy):
    gx = [int(v) for v in gx]
    gy = [int(v) for v in gy]
    return (sum(x * x for x in gx), sum(x * y for x, y in zip(gx, gy)), sum(y * y for y in gy))


def _random_tensors(rng, n):
    """Structure tensors of (2 br + 1)^2 raw Scharr samples in [-4080, 4080]:
    isotropic, near rank one (an edge: gy ~ k gx), near isotropic, extreme."""
    out = []
    for i in range(n):
        br = 1 if i % 2 == 0 else 2
        m = (2 * br + 1) ** 2
        kind = i % 4
        gx = rng.integers(-4080, 4081, m)
        if kind == 0:
            gy = rng.integers(-4080, 4081, m)
        elif kind == 1:
            k = rng.uniform(-3, 3)
            gy = np.clip(np.round(k * gx) + rng.integers(-2, 3, m), -4080, 4080)
        elif kind == 2:
            gy = np.clip(np.round(gx * rng.uniform(0.9, 1.1)) + rng.integers(-300, 301, m), -4080, 4080)
            gx = np.clip(gx + rng.integers(-300, 301, m), -4080, 4080)
        else:
            gx = rng.choice([-4080, 4080], m)
            gy = rng.choice([-4080, 4080], m)
        out.append(_tensor(gx, gy))
    return out


def _score_within_bound(score, a, b, c):
    return abs(score - _exact_lmin(a, b, c)) <= BOUND * (a + c)


def test_fp32_score_is_exact_lambda_min_within_its_rounding_bound():
    rng = np.random.Generator(np.random.PCG64(2024))
    worst = 0.0
    for a, b, c in _random_tensors(rng, 4000):
        lam = _exact_lmin(a, b, c)
        s = oracle.gftt_score(a, b, c)
        assert abs(s - lam) <= BOUND * (a + c), (a, b, c, s, lam)
        worst = max(worst, abs(s - lam) / (U * (a + c)))
    assert worst > 0.05  # the bound is not vacuous: real rounding is seen


def test_plausible_slips_in_the_score_violate_the_bound():
    """The bound separates the stated sequence from plausible slips: 4 b^2
    written as b^2, the root added instead of subtracted, or a - c replaced by
    a + c each fall outside it on realistic tensors."""
    f = np.float32
    rng = np.random.Generator(np.random.PCG64(7))
    ts = _random_tensors(rng, 200)

    def seq(a, b, c, four=4.0, sign=-1.0, diff=True):
        fa, fb, fc = f(a), f(b), f(c)
        d = f(fa - fc) if diff else f(fa + fc)
        r = np.sqrt(f(f(d * d) + f(f(four) * f(fb * fb))))
        return max(float(f(f(0.5) * f(f(fa + fc) + f(sign) * r))), 0.0)

    assert all(_score_within_bound(seq(a, b, c), a, b, c) for a, b, c in ts)  # the stated sequence
    for slip in (dict(four=1.0), dict(sign=1.0), dict(diff=False)):
        assert not all(_score_within_bound(seq(a, b, c, **slip), a, b, c) for a, b, c in ts), slip


def _box_tensors(gx, gy, br):
    """Exact (a, b, c) of every pixel: (2 br + 1)^2 box sums of the raw Scharr
    products with reflect-101 borders (numpy's 'reflect' mode)."""
    gx, gy = gx.astype(np.int64), gy.astype(np.int64)
    h, w = gx.shape

    def box(v):
        p = np.pad(v, br, mode="reflect")
        out = np.zeros_like(v)
        for j in range(2 * br + 1):
            for i in range(2 * br + 1):
                out += p[j:j + h, i:i + w]
        return out

    return box(gx * gx), box(gx * gy), box(gy * gy)


def _select(s, quality, nms, border, min_dist, max_corners, mask=None):
    """Brute-force Shi-Tomasi selection on a score map (the rules of the
    oracle's reading): threshold quality * max and > 0, border, local maximum
    of the (2 nms + 1)^2 window (out-of-image neighbours ignored, equal
    scores resolved to the smaller row-major index), greedy minimum distance
    in (score descending, index ascending) order, at most max_corners."""
    h, w = s.shape
    thr = quality * s.max()
    pad = np.pad(s, nms, constant_values=-np.inf)
    wmax = np.lib.stride_tricks.sliding_window_view(pad, (2 * nms + 1, 2 * nms + 1)).max(axis=(2, 3))
    cand = []
    ys, xs = np.nonzero((s >= thr) & (s > 0) & (s >= wmax))
    for y, x in zip(ys, xs):
        if y < border or y >= h - border or x < border or x >= w - border:
            continue
        ok = True
        for j in range(-nms, nms + 1):
            for i in range(-nms, nms + 1):
                yy, xx = y + j, x + i
                if (i or j) and 0 <= yy < h and 0 <= xx < w and s[yy, xx] == s[y, x] and yy * w + xx < y * w + x:
                    ok = False
        if ok:
            cand.append(int(y * w + x))
    cand.sort(key=lambda k: (-s.flat[k], k))
    kept = []
    for k in cand:
        if len(kept) >= max_corners:
            break
        y, x = divmod(k, w)
        if all((x - kx) ** 2 + (y - ky) ** 2 >= min_dist * min_dist for kx, ky in kept):
            kept.append((x, y))
    return np.array(kept, np.int64).reshape(-1, 2), cand, thr


@pytest.mark.parametrize("prm", [(0.01, 4, 10, 10, 150, 1), (0.01, 2, 5, 5, 1000, 1), (0.02, 3, 8, 8, 400, 2)])
def test_fp32_selection_equals_exact_selection(prm):
    """On a seeded 752x480 texture the oracle's corners (FP32 scores) are the
    corners of the same rules on the exact FP64 eigenvalue, except where a
    decision is a close call: two candidates whose exact scores lie within
    the rounding bound of each other, or a score within it of the quality
    threshold.  The first difference, if any, must be such a close call."""
    quality, nms, border, min_dist, max_corners, br = prm
    img = synth.make_config1(1).I
    p = oracle.build_pyramid(img, 1)
    a, b, c = _box_tensors(p.gx[0], p.gy[0], br)
    det = (a * c - b * b).astype(np.float64)  # exact integers below 2^53 after the subtraction
    af, bf, cf = a.astype(np.float64), b.astype(np.float64), c.astype(np.float64)
    lmax = (af + cf) / 2 + np.sqrt(((af - cf) / 2) ** 2 + bf * bf)
    with np.errstate(invalid="ignore", divide="ignore"):
        lam = np.maximum(np.where(lmax > 0, det / lmax, 0.0), 0.0)
    bound = BOUND * (af + cf)
    xy, sc = oracle.gftt(p.gx[0], p.gy[0], max_corners, quality, min_dist, nms, br, border)
    exact, cand, thr = _select(lam, quality, nms, border, min_dist, max_corners)
    # the oracle's scores are the exact ones within the bound
    h, w = lam.shape
    idx = xy[:, 1] * w + xy[:, 0]
    assert np.all(np.abs(sc.astype(np.float64) - lam.flat[idx]) <= bound.flat[idx])
    if np.array_equal(xy, exact):
        return
    k = next(i for i in range(min(len(xy), len(exact)) + 1)
             if i == min(len(xy), len(exact)) or not np.array_equal(xy[i], exact[i]))
    suspects = [int(q[1] * w + q[0]) for q in (xy[k:k + 1].tolist() + exact[k:k + 1].tolist())]
    thr_err = BOUND * (af + cf).flat[int(np.argmax(lam))] * quality

    def close(q):
        if abs(lam.flat[q] - thr) <= bound.flat[q] + thr_err:
            return True
        near = [o for o in cand if abs(lam.flat[o] - lam.flat[q]) <= bound.flat[o] + bound.flat[q] and o != q]
        y, x = divmod(q, w)
        win = lam[max(0, y - nms):y + nms + 1, max(0, x - nms):x + nms + 1]
        return bool(near) or np.any((np.abs(win - lam.flat[q]) <= bound.flat[q] * 2) & (win != lam.flat[q]))

    assert any(close(q) for q in suspects), f"first difference at {k} is not a close call"
