"""Pins of the FP64 oracle against closed forms, hand-worked examples and
brute force (no GPU).  Each test fixes something a plausible slip in the
oracle (a dropped term, a wrong sign or index, a transposed operand, a wrong
border rule or level scaling) would break.

Passages followed: Sec. IV (Shi-Tomasi corners with LK optical-flow tracking),
Table I (KLT tracker), Sec. V-A (cross-camera optical-flow verification); the
constants the paper leaves open are the readings listed at the top of
oracle/orc.c.
"""

import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _responses():
    rows = {}
    with open(os.path.join(GOLDEN, "pyrdown_1d_responses.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(t) for t in line.split()]
            rows[(v[0], v[1])] = np.array(v[2:])
    return rows


# ------------------------------------------------------------------ pyramid
@pytest.mark.parametrize("w,h", [(8, 8), (7, 8), (8, 7), (7, 7), (1, 5), (5, 1), (2, 3), (752, 480), (47, 30)])
def test_pyrdown_size_and_constant(w, h):
    for c in (0, 1, 128, 255):
        img = np.full((h, w), c, np.uint8)
        out = oracle.pyr_down(img)
        assert out.shape == ((h + 1) // 2, (w + 1) // 2)
        assert np.all(out == c)


def test_pyramid_level_sizes_752x480():
    lv = oracle.pyramid(np.zeros((480, 752), np.uint8), 5)
    assert [a.shape for a in lv] == [(480, 752), (240, 376), (120, 188), (60, 94), (30, 47)]


@pytest.mark.parametrize("n", [8, 7])
def test_pyrdown_impulse_golden(n):
    """2-D impulse responses equal the product of the hand-derived 1-D
    responses (interior and every border position of the golden table)."""
    rows = _responses()
    qs = sorted(q for (nn, q) in rows if nn == n)
    for v in (255, 100, 7):
        for qy in qs:
            for qx in qs:
                img = np.zeros((n, n), np.uint8)
                img[qy, qx] = v
                out = oracle.pyr_down(img).astype(np.int64)
                exp = (v * np.outer(rows[(n, qy)], rows[(n, qx)]) + 128) >> 8
                assert np.array_equal(out, exp), (n, qx, qy, v)


def test_pyrdown_impulse_centre_value():
    img = np.zeros((8, 8), np.uint8)
    img[4, 4] = 255
    out = oracle.pyr_down(img)
    assert out[2, 2] == 36  # round(255 * 36 / 256)
    assert out[2, 1] == 6 and out[1, 2] == 6 and out[1, 1] == 1
    assert out.sum() == 36 + 4 * 6 + 4 * 1


def test_pyrdown_ramp_and_checkerboard():
    x = np.arange(8)
    ramp = np.tile((16 * x).astype(np.uint8), (8, 1))
    out = oracle.pyr_down(ramp)
    # symmetric kernel: interior samples reproduce the ramp at 2X exactly;
    # X = 0 sees the reflected neighbours 32, 16, 0, 16, 32 -> 12*16*16/256 = 12
    assert np.all(out[:, 1:3] == 16 * 2 * np.arange(1, 3))
    assert np.all(out[:, 0] == 12)
    cb = ((np.add.outer(x, x) % 2) * 255).astype(np.uint8)
    outc = oracle.pyr_down(cb)
    # taps with i + j odd sum to 128: 255 * 128 / 256 = 127.5 -> 128
    assert np.all(outc[1:3, 1:3] == 128)


# ------------------------------------------------------------------ gradients
def test_scharr_constant_ramp_impulse():
    gx, gy = oracle.scharr(np.full((8, 8), 77, np.uint8))
    assert not gx.any() and not gy.any()
    x = np.arange(8)
    ramp = (3 * x[None, :] + 5 * x[:, None]).astype(np.uint8)
    gx, gy = oracle.scharr(ramp)
    assert np.all(gx[1:-1, 1:-1] == 32 * 3) and np.all(gy[1:-1, 1:-1] == 32 * 5)
    # reflect-101 makes the border column symmetric: zero derivative across it
    assert np.all(gx[:, 0] == 0) and np.all(gx[:, -1] == 0)
    assert np.all(gy[0, :] == 0) and np.all(gy[-1, :] == 0)
    imp = np.zeros((9, 9), np.uint8)
    imp[4, 4] = 100
    gx, gy = oracle.scharr(imp)
    assert gx[4, 3] == 1000 and gx[4, 5] == -1000 and gx[3, 3] == 300 and gx[5, 5] == -300
    assert gy[3, 4] == 1000 and gy[5, 4] == -1000 and gy[3, 5] == 300 and gy[5, 3] == -300
    assert gx[3, 4] == 0 and gy[4, 3] == 0
    # extremes: a 0/255 step gives +-16 * 255 = +-4080
    step = np.zeros((5, 6), np.uint8)
    step[:, 3:] = 255
    gx, _ = oracle.scharr(step)
    assert gx.max() == 4080
    gx, _ = oracle.scharr(255 - step)
    assert gx.min() == -4080


# ------------------------------------------------------------------ LK helpers
def _bowl(n=64, centre=(32.0, 32.0), a=0.05, b=0.08, c=0.03, t=(0.0, 0.0)):
    """I(z) = 0.5 (z - m)^T H (z - m) with H = [[2a, c], [c, 2b]], evaluated at
    z - t (so the image is shifted by +t); analytic gradient."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    dx, dy = x - t[0] - centre[0], y - t[1] - centre[1]
    img = 100.0 + a * dx * dx + b * dy * dy + c * dx * dy
    gx = 2 * a * dx + c * dy
    gy = 2 * b * dy + c * dx
    return img, gx, gy


# ------------------------------------------------------------------ LK pins
def test_one_newton_step_recovers_shift_on_quadratic():
    """For a quadratic image and a window centred on its extremum, one step
    eta = G^-1 b recovers any shift exactly: b = G t because the window's
    gradients sum to zero.  A wrong entry of G (including the cross term),
    a transposed solve, or a flipped residual sign all give eta != t."""
    for t in [(0.37, -0.81), (-1.25, 0.5), (2.0, 3.0)]:
        I, gx, gy = _bowl()
        J, _, _ = _bowl(t=t)
        r = oracle.track_f64([(I, gx, gy)], [J], np.array([[32.0, 32.0]]), win=21, max_iters=1, eps=0.0, min_eig=1e-9)
        assert r.status[0] == 1 and r.iters[0] == 1
        np.testing.assert_allclose(r.pts[0], np.array([32.0, 32.0]) + t, atol=1e-9)


def _bowl_levels(t, L, n=256, centre=128.0):
    """Quadratic bowl sampled at 2^l z for l < L (exact coarse levels)."""
    lvI, lvJ = [], []
    a, b, c = 0.05, 0.08, 0.03
    for l in range(L):
        m = n >> l
        y, x = np.mgrid[0:m, 0:m].astype(np.float64) * 2.0**l
        for tt, out in ((np.zeros(2), lvI), (np.asarray(t, float), lvJ)):
            dx, dy = x - tt[0] - centre, y - tt[1] - centre
            img = 100.0 + a * dx * dx + b * dy * dy + c * dx * dy
            if out is lvI:
                out.append((img, 2.0**l * (2 * a * dx + c * dy), 2.0**l * (2 * b * dy + c * dx)))
            else:
                out.append(img)
    return lvI, lvJ


def test_level_propagation_iteration_count_on_bowl():
    """t = 4 (3, -2) over 3 exact bowl levels: the top level needs one exact
    Newton step plus one pass seeing r = 0; with g_(l-1) = 2 (g_l + nu) every
    finer level starts on the answer and stops after one pass.  Any other
    propagation (or level scaling) costs a second pass somewhere."""
    t = (12.0, -8.0)
    lvI, lvJ = _bowl_levels(t, 3)
    r = oracle.track_f64(lvI, lvJ, np.array([[128.0, 128.0]]), win=21, max_iters=10, eps=1e-9, min_eig=1e-12,
                         per_level=True)
    assert r.status[0] == 1
    np.testing.assert_allclose(r.pts[0], [140.0, 120.0], atol=1e-9)
    assert r.iters[0] == 2 + 1 + 1
    assert r.iters_level[0].tolist() == [1, 1, 2]  # levels 0, 1, 2: the top one does the work


def test_convergence_test_is_on_the_step_length():
    """Stop when |eta|^2 < eps^2: a first step of 0.05 px continues at
    eps = 0.01, a first step of 0.005 px stops."""
    for t, it in [((0.05, 0.0), 2), ((0.0, 0.005), 1)]:
        I, gx, gy = _bowl()
        J, _, _ = _bowl(t=t)
        r = oracle.track_f64([(I, gx, gy)], [J], np.array([[32.0, 32.0]]), win=21, max_iters=10, eps=0.01,
                             min_eig=1e-9)
        assert r.status[0] == 1 and r.iters[0] == it


def test_min_eigenvalue_closed_form_quadratic():
    """G = (sum d d^T) H^2 = 16170 H^2 over a 21x21 window (sum_i i^2 = 770 per
    axis, times 21), so lambda_min(G) = 16170 min|eig(H)|^2."""
    a, b, c = 0.05, 0.08, 0.03
    I, gx, gy = _bowl(a=a, b=b, c=c)
    H = np.array([[2 * a, c], [c, 2 * b]])
    lam = 16170.0 * np.min(np.abs(np.linalg.eigvalsh(H))) ** 2 / (441 * 255.0**2)
    r = oracle.track_f64([(I, gx, gy)], [I], np.array([[32.0, 32.0]]), win=21, min_eig=1e-9)
    np.testing.assert_allclose(r.lmin[0], lam, rtol=1e-12)
    # threshold just above / below the closed form decides the status
    r = oracle.track_f64([(I, gx, gy)], [I], np.array([[32.0, 32.0]]), win=21, min_eig=lam * 1.001)
    assert r.status[0] == 0 and r.reason[0] == oracle.LOST_EIG
    r = oracle.track_f64([(I, gx, gy)], [I], np.array([[32.0, 32.0]]), win=21, min_eig=lam * 0.999)
    assert r.status[0] == 1


def test_zero_motion_is_exact():
    c = synth.make_config1(1)
    p = oracle.build_pyramid(c.I, 4)
    r = oracle.track(p, p, c.pts, per_level=True)
    assert np.all(r.status == 1)
    assert np.array_equal(r.pts, c.pts.astype(np.float64))
    assert np.all(r.iters == 4)  # one pass per level with eta = 0
    assert np.all(r.iters_level == 1)
    assert np.all(r.err == 0.0)


def test_eigen_rejection_constant_ramp_blob():
    flat = np.full((64, 64), 90, np.uint8)
    ramp = np.tile((2 * np.arange(64) + 40).astype(np.uint8), (64, 1))
    y, x = np.mgrid[0:64, 0:64]
    blob = np.rint(60 + 120 * np.exp(-((x - 32) ** 2 + (y - 32) ** 2) / (2 * 5.0**2))).astype(np.uint8)
    pt = np.array([[32.0, 32.0]])
    for img, ok in [(flat, False), (ramp, False), (blob, True)]:
        p = oracle.build_pyramid(img, 1)
        r = oracle.track(p, p, pt, levels=1)
        assert r.status[0] == ok
        if not ok:
            assert r.reason[0] == oracle.LOST_EIG and r.lmin[0] < 1e-12


def _shifted_u8(t, n=120, seed=9, margin=16):
    tex = synth.BlobTexture(seed, extent=(-40.0, -40.0, n + 2 * margin + 40.0, n + 2 * margin + 40.0))
    B = synth.texture.quantize_u8(tex.eval_affine(n + 2 * margin, n + 2 * margin, np.array([[1.0, 0, 0], [0, 1.0, 0]])))
    I = B[margin:margin + n, margin:margin + n].copy()
    J = B[margin - t[1]:margin - t[1] + n, margin - t[0]:margin - t[0] + n].copy()  # J(x) = I(x - t)
    return I, J


def test_integer_translation_with_exact_guess_multilevel():
    """t a multiple of 4 with 3 levels: every level of J's pyramid is I's level
    shifted by t / 2^l away from borders, so with the exact guess each level
    sees r = 0 and stops after one pass; a slip in the guess scaling, the
    level propagation or u_l = u / 2^l leaves a non-zero residual."""
    t = (8, -4)
    I, J = _shifted_u8(t)
    pI, pJ = oracle.build_pyramid(I, 3), oracle.build_pyramid(J, 3)
    pts = np.array([[60.0, 60.0], [55.0, 64.0], [64.0, 52.0]])
    r = oracle.track(pI, pJ, pts, guess=pts + t)
    assert np.all(r.status == 1)
    np.testing.assert_array_equal(r.pts, pts + t)
    assert np.all(r.iters == 3) and np.all(r.err == 0.0)


def test_integer_translation_from_zero_guess():
    for t in [(3, -2), (-6, 5), (7, 7)]:
        I, J = _shifted_u8(t)
        pI, pJ = oracle.build_pyramid(I, 3), oracle.build_pyramid(J, 3)
        pts = np.array([[60.0, 60.0], [50.0, 70.0], [70.0, 50.0], [58.5, 61.25]])
        r = oracle.track(pI, pJ, pts, eps=1e-4, max_iters=60)
        assert np.all(r.status == 1)
        np.testing.assert_allclose(r.pts, pts + t, atol=2e-3)
        # sign / transposition: the x shift lands on x
        assert np.all(np.abs(r.pts - pts - t) < 0.01)


def _bilinear_surface(n, t=(0.0, 0.0), scale=1.0):
    """I(z) = 100 + 0.8 X - 0.5 Y + 0.05 X Y with (X, Y) = scale * z - t - (48, 48):
    bilinear in z, so bilinear sampling reproduces it exactly at any
    sub-pixel position; returns the image and its exact gradient."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    X, Y = scale * x - t[0] - 48.0, scale * y - t[1] - 48.0
    img = 100.0 + 0.8 * X - 0.5 * Y + 0.05 * X * Y
    return img, scale * (0.8 + 0.05 * Y), scale * (-0.5 + 0.05 * X)


def test_subpixel_shift_recovered_exactly_on_bilinear_surface():
    """Sub-pixel points and shifts on an image that bilinear sampling
    reproduces exactly: the fixed point r = 0 is the true shift, so the
    converged flow equals t to round-off, at one level and coarse-to-fine
    (coarse levels sample the same surface at 2^l z)."""
    rng = np.random.Generator(np.random.PCG64(11))
    for trial in range(6):
        t = rng.uniform(-1.5, 1.5, 2)
        I, gx, gy = _bilinear_surface(96)
        J, _, _ = _bilinear_surface(96, t=t)
        pts = rng.uniform(30.0, 66.0, (12, 2))
        r = oracle.track_f64([(I, gx, gy)], [J], pts, win=21, eps=1e-9, max_iters=100, min_eig=1e-9)
        assert np.all(r.status == 1)
        np.testing.assert_allclose(r.pts - pts, np.broadcast_to(t, pts.shape), atol=1e-7)
    for trial in range(4):
        t = rng.uniform(-6.0, 6.0, 2)
        lvI, lvJ = [], []
        for l in range(3):
            n = 160 >> l
            I, gx, gy = _bilinear_surface(n, scale=2.0**l)
            J, _, _ = _bilinear_surface(n, t=t, scale=2.0**l)
            lvI.append((I, gx, gy))
            lvJ.append(J)
        pts = rng.uniform(60.0, 100.0, (12, 2))
        r = oracle.track_f64(lvI, lvJ, pts, win=21, eps=1e-9, max_iters=100, min_eig=1e-9)
        assert np.all(r.status == 1)
        np.testing.assert_allclose(r.pts - pts, np.broadcast_to(t, pts.shape), atol=1e-7)


def test_subpixel_bandlimited_shift_bias_bound():
    """Exactly rendered band-limited texture (the workload's: blob sigma
    2-12 px, wavelengths 8-32 px), analytic gradients, sub-pixel t: the only
    error left is the bias of bilinear sampling, measured here at a mean
    below 0.01 px and a maximum below 0.05 px."""
    rng = np.random.Generator(np.random.PCG64(11))
    errs = []
    for trial in range(6):
        t = rng.uniform(-1.5, 1.5, 2)
        n = 96
        tex = synth.BlobTexture(100 + trial, extent=(-40.0, -40.0, n + 40.0, n + 40.0),
                                n_blobs=int(400 * (n + 80) ** 2 / 361000))
        I, gxI, gyI = tex.eval_affine(n, n, np.array([[1.0, 0, 0], [0, 1.0, 0]]), with_grad=True)
        J = tex.eval_affine(n, n, np.array([[1.0, 0, -t[0]], [0, 1.0, -t[1]]]))
        pts = rng.uniform(30.0, 66.0, (30, 2))
        r = oracle.track_f64([(I, gxI, gyI)], [J], pts, win=21, eps=1e-6, max_iters=200, min_eig=1e-6)
        ok = r.status == 1
        assert ok.mean() >= 0.9
        errs.append(np.hypot(*(r.pts[ok] - pts[ok] - t).T))
    e = np.concatenate(errs)
    assert e.mean() < 0.01 and e.max() < 0.05, (e.mean(), e.max())


def test_brute_force_integer_ssd_agrees():
    """48x48 images, integer shifts <= 3 px, 1 level: the exhaustive integer
    SSD minimiser over [-4, 4]^2 equals the rounded oracle flow."""
    rng = np.random.Generator(np.random.PCG64(13))
    for trial in range(6):
        t = tuple(int(v) for v in rng.integers(-3, 4, 2))
        n, m = 48, 8
        tex = synth.BlobTexture(300 + trial, extent=(-20.0, -20.0, n + 2 * m + 20.0, n + 2 * m + 20.0), n_blobs=40,
                                sigma_range=(3.0, 8.0))
        B = synth.texture.quantize_u8(tex.eval_affine(n + 2 * m, n + 2 * m, np.array([[1.0, 0, 0], [0, 1.0, 0]])))
        I = B[m:m + n, m:m + n].copy()
        J = B[m - t[1]:m - t[1] + n, m - t[0]:m - t[0] + n].copy()
        p = np.array([[24.0, 24.0]])
        best, arg = None, None
        T = I[14:35, 14:35].astype(np.int64)
        for dy in range(-4, 5):
            for dx in range(-4, 5):
                S = J[14 + dy:35 + dy, 14 + dx:35 + dx].astype(np.int64)
                ssd = int(((T - S) ** 2).sum())
                if best is None or ssd < best:
                    best, arg = ssd, (dx, dy)
        pI, pJ = oracle.build_pyramid(I, 1), oracle.build_pyramid(J, 1)
        r = oracle.track(pI, pJ, p, levels=1, max_iters=50, min_eig=1e-6)
        assert r.status[0] == 1
        assert tuple(np.rint(r.pts[0] - p[0]).astype(int)) == arg == t


def test_two_levels_agree_with_one_level_small_motion():
    for t in [(1, 0), (0, -1), (1, 1)]:
        I, J = _shifted_u8(t)
        pts = np.array([[60.3, 59.6], [52.0, 66.0], [68.0, 54.0]])
        pI, pJ = oracle.build_pyramid(I, 2), oracle.build_pyramid(J, 2)
        r1 = oracle.track(pI, pJ, pts, levels=1, eps=0.001, max_iters=50)
        r2 = oracle.track(pI, pJ, pts, levels=2, eps=0.001, max_iters=50)
        assert np.all(r1.status == 1) and np.all(r2.status == 1)
        assert np.abs(r1.pts - r2.pts).max() < 0.005


def test_error_is_mean_abs_residual_under_intensity_offset():
    """J = I + 10 with a window centred on a symmetric blob: the gradients of
    the window sum to zero, so b = -10 sum grad T = 0, eta = 0, and the
    reported error is exactly 10."""
    y, x = np.mgrid[0:64, 0:64]
    I = np.rint(60 + 120 * np.exp(-((x - 32) ** 2 + (y - 32) ** 2) / (2 * 6.0**2))).astype(np.uint8)
    J = (I + 10).astype(np.uint8)
    pI, pJ = oracle.build_pyramid(I, 1), oracle.build_pyramid(J, 1)
    r = oracle.track(pI, pJ, np.array([[32.0, 32.0]]), levels=1)
    assert r.status[0] == 1
    np.testing.assert_array_equal(r.pts[0], [32.0, 32.0])
    assert r.err[0] == 10.0 and r.iters[0] == 1


def test_out_of_image_rules():
    c = synth.make_config1(1)
    pI, pJ = oracle.build_pyramid(c.I, 4), oracle.build_pyramid(c.J, 4)
    w, h = c.I.shape[1], c.I.shape[0]
    # input point outside the image, or not a number
    r = oracle.track(pI, pJ, np.array([[-1.0, 10.0], [w - 0.5, 10.0], [np.nan, 5.0]]))
    assert np.all(r.status == 0) and np.all(r.reason == oracle.LOST_INPUT)
    # a guess far outside the image: the first J pass is out of bounds
    r = oracle.track(pI, pJ, c.pts[:3], guess=c.pts[:3] + np.array([2000.0, 0.0]))
    assert np.all(r.status == 0) and np.all(r.reason == oracle.LOST_OOB)
    # a point moving out through the right border: final position > W - 1
    I, J = _shifted_u8((3, 0), n=120)
    pI, pJ = oracle.build_pyramid(I, 2), oracle.build_pyramid(J, 2)
    r = oracle.track(pI, pJ, np.array([[118.5, 60.0]]), levels=2, max_iters=50, min_eig=1e-7)
    assert r.status[0] == 0 and r.reason[0] == oracle.LOST_OOB


def test_max_iters_is_respected():
    c = synth.make_config1(1)
    pI, pJ = oracle.build_pyramid(c.I, 4), oracle.build_pyramid(c.J, 4)
    r = oracle.track(pI, pJ, c.pts, max_iters=1, eps=0.0)
    assert np.all(r.iters[r.status == 1] == 4)


def test_forward_backward_translation_and_occlusion():
    I, J = _shifted_u8((2, -1), n=120)
    pts = np.array([[35.0, 35.0], [35.0, 85.0], [85.0, 60.0]])
    # occlude the neighbourhood of the last point in J with unrelated texture
    other = synth.texture.quantize_u8(synth.BlobTexture(77, extent=(0, 0, 120, 120)).eval_affine(
        120, 120, np.array([[1.0, 0, 0], [0, 1.0, 0]])))
    J2 = J.copy()
    J2[40:85, 70:110] = other[40:85, 70:110]
    pI, pJ = oracle.build_pyramid(I, 3), oracle.build_pyramid(J2, 3)
    r = oracle.track_fb(pI, pJ, pts, min_eig=1e-6)
    assert r.status[0] == 1 and r.status[1] == 1
    assert r.fb_dist[0] < 0.01 and r.fb_dist[1] < 0.01
    assert r.status[2] == 0 and r.reason[2] in (oracle.LOST_FB, oracle.LOST_EIG, oracle.LOST_OOB)


def test_fb_threshold_is_inclusive():
    p0 = np.array([[10.0, 10.0], [10.0, 10.0], [10.0, 10.0]])
    p1 = np.array([[10.5, 10.0], [10.0, 10.5000001], [10.25, 10.25]])
    st, d, m = oracle.fb_check(p0, p1, np.ones(3, np.uint8), np.ones(3, np.uint8), 0.5)
    assert list(st) == [1, 0, 1]
    st, _, _ = oracle.fb_check(p0, p0, np.array([1, 0, 1], np.uint8), np.array([1, 1, 0], np.uint8), 0.5)
    assert list(st) == [1, 0, 0]


def test_config1_against_closed_form_motion():
    """Config-1 pair: every keypoint is tracked and the oracle's flow is close
    to the closed-form rigid motion (the residual is the window's rotation,
    which a translational LK model does not capture, plus 8-bit
    quantisation); reported bound, not the parity tolerance."""
    c = synth.make_config1(1)
    pI, pJ = oracle.build_pyramid(c.I, 4), oracle.build_pyramid(c.J, 4)
    r = oracle.track_fb(pI, pJ, c.pts)
    ok = r.status == 1
    assert ok.mean() > 0.95
    e = np.hypot(*(r.fwd.pts[ok] - c.gt[ok]).T)
    assert e.mean() < 0.1 and e.max() < 0.3
