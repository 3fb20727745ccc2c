"""Pins of the oracle's Shi-Tomasi detector (no GPU): closed-form scores,
corners of synthetic squares found where they are, and the selection rules
(minimum distance, priority order, mask, cap, non-maximum suppression)."""

import numpy as np

import oracle
import synth


def test_score_closed_forms():
    assert oracle.gftt_score(10, 0, 4) == 4.0  # diagonal: the smaller entry
    assert oracle.gftt_score(4, 0, 10) == 4.0
    assert oracle.gftt_score(5, 5, 5) == 0.0  # rank one (b^2 = a c): an edge
    assert oracle.gftt_score(9, 6, 4) == 0.0
    assert oracle.gftt_score(0, 0, 0) == 0.0
    # [[2, 1], [1, 2]] has eigenvalues 1 and 3
    assert oracle.gftt_score(2, 1, 2) == 1.0


def _squares(n=160, side=12, step=40, lo=20, hi=200):
    img = np.full((n, n), lo, np.uint8)
    corners = []
    for y0 in range(20, n - side - 10, step):
        for x0 in range(20, n - side - 10, step):
            img[y0:y0 + side, x0:x0 + side] = hi
            corners += [(x0, y0), (x0 + side - 1, y0), (x0, y0 + side - 1), (x0 + side - 1, y0 + side - 1)]
    return img, np.array(corners, float)


def test_square_corners_are_found():
    img, true = _squares()
    p = oracle.build_pyramid(img, 1)
    xy, sc = oracle.gftt(p.gx[0], p.gy[0], max_corners=1000, quality=0.05, min_dist=5, nms_radius=2, border=4)
    d = np.hypot(xy[:, None, 0] - true[None, :, 0], xy[:, None, 1] - true[None, :, 1])
    assert np.all(d.min(axis=1) <= 1.5), "a detection away from every square corner"
    assert np.all(d.min(axis=0) <= 1.5), "a square corner without a detection"
    assert len(xy) == len(true)


def test_selection_rules():
    c = synth.make_config1(1)
    p = oracle.build_pyramid(c.I, 1)
    xy, sc = oracle.gftt(p.gx[0], p.gy[0], max_corners=400, quality=0.01, min_dist=12, nms_radius=4, border=10)
    assert len(xy) == 400
    dd = ((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(dd, 10 ** 9)
    assert dd.min() >= 12 * 12
    assert np.all(np.diff(sc) <= 0)  # priority order
    assert xy[:, 0].min() >= 10 and xy[:, 1].min() >= 10
    assert xy[:, 0].max() <= c.I.shape[1] - 11 and xy[:, 1].max() <= c.I.shape[0] - 11
    # the cap keeps a prefix of the uncapped greedy selection
    xy2, _ = oracle.gftt(p.gx[0], p.gy[0], max_corners=8192, quality=0.01, min_dist=12, nms_radius=4, border=10)
    assert len(xy2) > 400 and np.array_equal(xy2[:400], xy)
    # a mask removes everything within min_dist of its points
    mask = xy[:50].astype(np.float64) + 0.25
    xy3, _ = oracle.gftt(p.gx[0], p.gy[0], max_corners=400, quality=0.01, min_dist=12, nms_radius=4, border=10,
                         mask=mask)
    dm = ((xy3[:, None, :] - mask[None, :, :]) ** 2).sum(-1)
    assert dm.min() >= 144


def test_nms_separates_maxima():
    c = synth.make_config1(2)
    p = oracle.build_pyramid(c.I, 1)
    xy, sc = oracle.gftt(p.gx[0], p.gy[0], max_corners=8192, quality=0.0, min_dist=1, nms_radius=3, border=3)
    cheb = np.maximum(np.abs(xy[:, None, 0] - xy[None, :, 0]), np.abs(xy[:, None, 1] - xy[None, :, 1]))
    np.fill_diagonal(cheb, 99)
    assert cheb.min() > 3
