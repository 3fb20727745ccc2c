"""Pyramidal LK (K3) and forward-backward check (K4) through the C ABI,
compared with the FP64 oracle point by point on the same seeded inputs."""

import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


def _vt():
    import paper_2607_01757_gb300 as vt

    return vt


def _gpu_track(I, J, pts, prm, fb=False, guess=None, grad=1, stream=None):
    import torch

    vt = _vt()
    pI = vt.vt_pyramid_build_grad(I, prm.levels, grad)
    pJ = vt.vt_pyramid_build_grad(J, prm.levels, grad)
    n = len(pts)
    d_in = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    d_g = None if guess is None else torch.from_numpy(np.ascontiguousarray(guess, np.float32)).cuda()
    out = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    err = torch.zeros(n, dtype=torch.float32, device="cuda")
    rs = torch.zeros(n, dtype=torch.uint8, device="cuda")
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    lm = torch.zeros(n, dtype=torch.float32, device="cuda")
    if fb:
        vt.vt_klt_track_fb(pI, pJ, d_in, prm, out, st, err, reason=rs, iters=it, lmin=lm)
    else:
        vt.vt_klt_track_ex(pI, pJ, d_in, prm, out, st, err, pts_guess=d_g, reason=rs, iters=it, lmin=lm)
    torch.cuda.synchronize()
    res = dict(pts=out.cpu().numpy(), status=st.cpu().numpy(), err=err.cpu().numpy(), reason=rs.cpu().numpy(),
               iters=it.cpu().numpy(), lmin=lm.cpu().numpy())
    pI.free()
    pJ.free()
    return res


def _ref(I, J, pts, prm, fb=False, guess=None):
    pI, pJ = oracle.build_pyramid(I, prm.levels), oracle.build_pyramid(J, prm.levels)
    if fb:
        return oracle.track_fb(pI, pJ, pts, prm.win, prm.levels, prm.max_iters, prm.eps, prm.min_eig, prm.fb_thr)
    return oracle.track(pI, pJ, pts, prm.win, prm.levels, prm.max_iters, prm.eps, prm.min_eig, guess=guess)


def _check(g, r, label, fb=False):
    st = compare(g["pts"], g["status"], g["reason"], r, label)
    both = (g["status"] == 1) & (r.status == 1)
    err_ref = r.fwd.err if fb else r.err
    np.testing.assert_allclose(g["err"][both], err_ref[both], rtol=2e-3, atol=2e-3)
    return st


@pytest.fixture(scope="module")
def cfg1():
    return synth.make_config1(1)


def test_config1_forward(cfg1):
    vt = _vt()
    prm = vt.KltParams(win=21, levels=4, max_iters=30, eps=0.01, fb_thr=0.5)
    g = _gpu_track(cfg1.I, cfg1.J, cfg1.pts, prm)
    r = _ref(cfg1.I, cfg1.J, cfg1.pts, prm)
    st = _check(g, r, "config1 forward")
    assert st["tracked_ref"] >= 140
    agree = (g["status"] == 1) & (r.status == 1) & (r.margin.min(axis=1) > 1e-3)
    # iteration counts agree wherever no convergence decision was marginal
    assert (g["iters"][agree] == r.iters[agree]).mean() > 0.98
    np.testing.assert_allclose(g["lmin"][agree], r.lmin[agree], rtol=1e-4)


def test_config1_forward_backward(cfg1):
    vt = _vt()
    prm = vt.KltParams(win=21, levels=4, max_iters=30, eps=0.01, fb_thr=0.5)
    g = _gpu_track(cfg1.I, cfg1.J, cfg1.pts, prm, fb=True)
    r = _ref(cfg1.I, cfg1.J, cfg1.pts, prm, fb=True)
    _check(g, r, "config1 fb", fb=True)
    same = g["status"] == r.status
    assert np.all(g["reason"][same & (r.status == 0)] == r.reason[same & (r.status == 0)])


def test_fused_fb_equals_separate_calls(cfg1):
    """vt_klt_track_fb == vt_klt_track_ex forward, _ex backward, vt_fb_check."""
    import torch

    vt = _vt()
    prm = vt.KltParams(win=21, levels=4, max_iters=30, eps=0.01, fb_thr=0.5)
    pI = vt.vt_pyramid_build_grad(cfg1.I, 4)
    pJ = vt.vt_pyramid_build_grad(cfg1.J, 4)
    n = len(cfg1.pts)
    p0 = torch.from_numpy(cfg1.pts).cuda()
    f_out, b_out = torch.zeros_like(p0), torch.zeros_like(p0)
    f_st, b_st, fb_st = (torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(3))
    vt.vt_klt_track_ex(pI, pJ, p0, prm, f_out, f_st)
    vt.vt_klt_track_ex(pJ, pI, f_out, prm, b_out, b_st)
    vt.vt_fb_check(p0, b_out, f_st, b_st, prm.fb_thr, fb_st)
    u_out, u_st = torch.zeros_like(p0), torch.zeros(n, dtype=torch.uint8, device="cuda")
    vt.vt_klt_track_fb(pI, pJ, p0, prm, u_out, u_st)
    torch.cuda.synchronize()
    assert torch.equal(u_st, fb_st)
    ok = u_st.bool()
    assert (u_out[ok] - f_out[ok]).abs().max().item() <= 1e-5


@pytest.mark.parametrize("with_guess", [False, True])
def test_plain_klt_track_entry_point(cfg1, with_guess):
    """vt_klt_track, the plain call of the boundary (no diagnostics, default
    eigenvalue threshold 1e-4), on config 1 with and without pts_guess (the
    ground-truth positions offset by a seeded error of up to 2 px): equal to
    vt_klt_track_ex on the same inputs bit for bit, and within parity of the
    oracle (the status rule reads the reasons _ex reports)."""
    import torch

    vt = _vt()
    pI = vt.vt_pyramid_build_grad(cfg1.I, 4)
    pJ = vt.vt_pyramid_build_grad(cfg1.J, 4)
    n = len(cfg1.pts)
    p0 = torch.from_numpy(np.ascontiguousarray(cfg1.pts, np.float32)).cuda()
    guess_h = None
    g = None
    if with_guess:
        rng = np.random.Generator(np.random.PCG64(71))
        guess_h = (cfg1.gt + rng.uniform(-2.0, 2.0, cfg1.gt.shape)).astype(np.float32)
        g = torch.from_numpy(guess_h).cuda()
    out, st, err = torch.zeros((n, 2), device="cuda"), torch.zeros(n, dtype=torch.uint8, device="cuda"), \
        torch.zeros(n, device="cuda")
    vt.vt_klt_track(pI, pJ, p0, out, st, err, pts_guess=g, win=21, levels=4, max_iters=30, eps=0.01)
    prm = vt.KltParams(win=21, levels=4, max_iters=30, eps=0.01, min_eig=1e-4)
    o2, s2, e2 = torch.zeros_like(out), torch.zeros_like(st), torch.zeros_like(err)
    rs = torch.zeros(n, dtype=torch.uint8, device="cuda")
    vt.vt_klt_track_ex(pI, pJ, p0, prm, o2, s2, e2, pts_guess=g, reason=rs)
    torch.cuda.synchronize()
    assert torch.equal(st, s2) and torch.equal(out, o2) and torch.equal(err, e2)
    r = _ref(cfg1.I, cfg1.J, cfg1.pts, prm, guess=None if guess_h is None else guess_h.astype(np.float64))
    stats = compare(out.cpu().numpy(), st.cpu().numpy(), rs.cpu().numpy(), r, f"vt_klt_track guess={with_guess}")
    assert stats["tracked_ref"] >= 140, stats
    both = (st.cpu().numpy() == 1) & (r.status == 1)
    np.testing.assert_allclose(err.cpu().numpy()[both], r.err[both], rtol=2e-3, atol=2e-3)
    pI.free()
    pJ.free()


@pytest.mark.parametrize("win", [9, 15, 31])
def test_other_windows(cfg1, win):
    vt = _vt()
    prm = vt.KltParams(win=win, levels=4, max_iters=30, eps=0.01, fb_thr=0.5,
                       min_eig=1e-4 if win >= 15 else 5e-5)
    g = _gpu_track(cfg1.I, cfg1.J, cfg1.pts[:97], prm, fb=True)
    r = _ref(cfg1.I, cfg1.J, cfg1.pts[:97], prm, fb=True)
    _check(g, r, f"win {win}", fb=True)


@pytest.mark.parametrize("n", [0, 1, 3, 5, 37])
def test_ragged_point_counts(cfg1, n):
    vt = _vt()
    prm = vt.KltParams()
    pts = cfg1.pts[:n]
    if n == 0:
        import torch

        pI = vt.vt_pyramid_build_grad(cfg1.I, 4)
        e = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
        s = torch.zeros(0, dtype=torch.uint8, device="cuda")
        vt.vt_klt_track_ex(pI, pI, e, prm, e, s)
        vt.vt_klt_track_fb(pI, pI, e, prm, e, s)
        return
    g = _gpu_track(cfg1.I, cfg1.J, pts, prm)
    r = _ref(cfg1.I, cfg1.J, pts, prm)
    _check(g, r, f"n={n}")


def test_zero_motion_and_degenerate_points(cfg1):
    vt = _vt()
    prm = vt.KltParams()
    w, h = cfg1.I.shape[1], cfg1.I.shape[0]
    pts = np.concatenate([cfg1.pts[:20], np.array([[0.0, 0.0], [w - 1.0, h - 1.0], [-0.5, 10.0], [w + 3.0, 5.0],
                                                   [np.nan, 3.0], [5.0, 5.0], [w - 2.0, 100.0]], np.float32)])
    g = _gpu_track(cfg1.I, cfg1.I, pts, prm)
    r = _ref(cfg1.I, cfg1.I, pts, prm)
    _check(g, r, "zero motion / border points")
    ok = r.status == 1
    assert np.array_equal(g["pts"][ok], pts[ok])  # I == J: flow is exactly zero
    assert np.all(g["reason"][[22, 23, 24]] == vt.VT_LOST_INPUT)
    # flat image: every point is rejected by the eigenvalue test
    flat = np.full_like(cfg1.I, 77)
    g = _gpu_track(flat, flat, cfg1.pts[:8], prm)
    assert np.all(g["status"] == 0) and np.all(g["reason"] == vt.VT_LOST_EIG)


def test_guess_and_iteration_cap(cfg1):
    vt = _vt()
    prm = vt.KltParams(max_iters=1, eps=0.0)
    g = _gpu_track(cfg1.I, cfg1.J, cfg1.pts, prm, guess=cfg1.gt.astype(np.float32))
    r = _ref(cfg1.I, cfg1.J, cfg1.pts, prm, guess=cfg1.gt)
    _check(g, r, "guess + max_iters=1")
    assert np.all(g["iters"][g["status"] == 1] == 4)
    far = cfg1.pts[:5] + np.array([3000.0, 0.0], np.float32)
    g = _gpu_track(cfg1.I, cfg1.J, cfg1.pts[:5], vt.KltParams(), guess=far)
    assert np.all(g["status"] == 0) and np.all(g["reason"] == vt.VT_LOST_OOB)


def test_deterministic_repeat(cfg1):
    vt = _vt()
    prm = vt.KltParams()
    a = _gpu_track(cfg1.I, cfg1.J, cfg1.pts, prm, fb=True)
    b = _gpu_track(cfg1.I, cfg1.J, cfg1.pts, prm, fb=True)
    for k in ("pts", "status", "err", "iters"):
        assert np.array_equal(a[k], b[k])


def test_fb_check_kernel():
    import torch

    vt = _vt()
    p0 = torch.tensor([[10.0, 10.0], [10.0, 10.0], [10.0, 10.0], [1.0, 1.0]], device="cuda")
    p1 = torch.tensor([[10.5, 10.0], [10.0, 10.5000005], [10.25, 10.25], [1.0, 1.0]], device="cuda")
    sf = torch.tensor([1, 1, 1, 0], dtype=torch.uint8, device="cuda")
    sb = torch.ones(4, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.uint8, device="cuda")
    vt.vt_fb_check(p0, p1, sf, sb, 0.5, out)
    torch.cuda.synchronize()
    ref, _, _ = oracle.fb_check(p0.cpu().numpy(), p1.cpu().numpy(), sf.cpu().numpy(), sb.cpu().numpy(), 0.5)
    assert out.cpu().numpy().tolist() == ref.tolist() == [1, 0, 1, 0]


def test_argument_errors():
    import torch

    vt = _vt()
    img = np.zeros((64, 64), np.uint8)
    p = vt.vt_pyramid_build(img, 3)
    e = torch.zeros((4, 2), device="cuda")
    s = torch.zeros(4, dtype=torch.uint8, device="cuda")
    # no stored gradients: the tracker computes them (no error)
    vt.vt_klt_track_ex(p, p, e, vt.KltParams(levels=3), e, s)
    vt.vt_gradients(p)
    for bad in (vt.KltParams(levels=4), vt.KltParams(levels=3, win=20), vt.KltParams(levels=3, win=11),
                vt.KltParams(levels=3, max_iters=0), vt.KltParams(levels=3, eps=-1.0)):
        with pytest.raises(vt.VTError):
            vt.vt_klt_track_ex(p, p, e, bad, e, s)
    q = vt.vt_pyramid_build_grad(img, 3, vt.VT_GRAD_F16)
    with pytest.raises(vt.VTError):  # fused FB needs one gradient type
        vt.vt_klt_track_fb(p, q, e, vt.KltParams(levels=3), e, s)


def test_near_singular_gradient_matrix_lambda_min():
    """λ_min of a nearly rank-one G.  Diagonal stripes of contrast 8 with a
    few pixels changed by one grey level keep every window sum of gradient
    products below 2^24, so the GPU's FP32 sums are exact integers equal to
    the oracle's: the only rounding left on the GPU is in λ_max (a square
    root) and in the determinant g11 g22 - g12^2.  For these points the
    determinant cancels by a factor ≥ 1e3 (a plain FP32 product difference
    would be off by far more than the bound below), and λ_min must match the
    oracle's exact one to 2e-6 relative."""
    vt = _vt()
    rng = np.random.default_rng(21)
    h, w = 96, 128
    y, x = np.mgrid[0:h, 0:w]
    img = (100 + 8 * ((x + y) % 6 < 3)).astype(np.uint8)
    flip = rng.random((h, w)) < 0.003
    img[flip] ^= 1
    pts = np.stack(np.meshgrid(np.arange(16, 112, 6), np.arange(16, 80, 6)), -1).reshape(-1, 2).astype(np.float32)
    prm = vt.KltParams(win=21, levels=1, max_iters=5, eps=0.01, min_eig=0.0)
    g = _gpu_track(img, img, pts, prm)
    r = _ref(img, img, pts, prm)
    # G from the oracle's integer gradients (raw Scharr) at the integer points
    rp = oracle.build_pyramid(img, 1)
    gx, gy = rp.gx[0].astype(np.int64), rp.gy[0].astype(np.int64)
    cancel, naive_err = [], []
    for px, py in pts.astype(int):
        wx = gx[py - 10:py + 11, px - 10:px + 11]
        wy = gy[py - 10:py + 11, px - 10:px + 11]
        a, b, c = int((wx * wx).sum()), int((wx * wy).sum()), int((wy * wy).sum())
        assert max(a, b, c) < 2 ** 24  # exact FP32 sums
        det = a * c - b * b
        naive = float(np.float32(np.float32(a) * np.float32(c)) - np.float32(np.float32(b) * np.float32(b)))
        cancel.append(a * c / det if det > 0 else np.inf)
        naive_err.append(abs(naive - det) / det if det > 0 else np.inf)
    cancel, naive_err = np.array(cancel), np.array(naive_err)
    sel = (r.status == 1) & (g["status"] == 1) & (cancel >= 1e3) & np.isfinite(cancel)
    assert sel.sum() >= 10, (sel.sum(), np.sort(cancel)[:10])
    # the bound below separates a compensated determinant from a plain one
    assert np.median(naive_err[sel]) > 1e-5
    np.testing.assert_allclose(g["lmin"][sel], r.lmin[sel], rtol=2e-6)
    assert (g["status"] == r.status).all()


def _stripes(w, h, theta, lam, amp, bumps, shift=(0.0, 0.0)):
    """Sinusoidal stripes across direction theta (period lam px, amplitude
    amp) plus small Gaussian bumps, evaluated exactly at pixel centres
    displaced by -shift (so the second frame is the scene moved by shift),
    rounded to uint8."""
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    x, y = x - shift[0], y - shift[1]
    img = 128 + amp * np.sin(2 * np.pi * (x * np.cos(theta) + y * np.sin(theta)) / lam)
    for bx, by, ba, bs in bumps:
        img += ba * np.exp(-((x - bx) ** 2 + (y - by) ** 2) / (2 * bs * bs))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


@pytest.mark.parametrize("theta_deg,lam,levels", [(0.0, 10.0, 1), (0.0, 16.0, 2), (20.0, 10.0, 1)])
def test_ill_conditioned_points_flow_against_oracle(theta_deg, lam, levels):
    """Points whose gradient matrix G has lambda_max / lambda_min > 1e5:
    high-contrast stripes whose only structure across them is a few small
    bumps (1-3 grey levels) and the uint8 rounding, the second frame the
    same scene moved by a sub-pixel shift.  The eigenvalue threshold is set
    low (1e-9) so these points are tracked, not rejected.  The tracker
    computes G, b and the Newton step in FP32 (the 2x2 determinant and the
    adjugate products by Kahan's compensated scheme, no FP64); its flow must
    still meet the usual tolerances against the FP64 oracle on exactly the
    points where the conditioning is worst.

    Where nothing across the stripes constrains the window, the flow is not
    determined by the data: the oracle's own result then moves by more than
    the tolerance when the input point moves by 1e-4 px (about 8-18 % of
    these points, mostly those that run out of iterations while sliding
    along the stripes), and no implementation short of repeating the
    oracle's arithmetic operation by operation can match it.  Such points
    are identified with the oracle alone (a second oracle run from the
    points moved by 1e-4 px; a result that moves by more than 1e-3 px is
    undetermined), counted, and left out of the comparison."""
    vt = _vt()
    rng = np.random.Generator(np.random.PCG64(int(theta_deg * 10 + lam)))
    w, h = 288, 208
    bumps = [(rng.uniform(0, w), rng.uniform(0, h), rng.choice([-1.0, 1.0]) * rng.uniform(1.0, 3.0),
              rng.uniform(1.0, 2.5)) for _ in range(70)]
    th = np.deg2rad(theta_deg)
    shift = (rng.uniform(-1.6, 1.6), rng.uniform(-1.6, 1.6))
    I = _stripes(w, h, th, lam, 120.0, bumps)
    J = _stripes(w, h, th, lam, 120.0, bumps, shift)
    pts = np.stack(np.meshgrid(np.arange(24, w - 24, 5), np.arange(24, h - 24, 5)), -1).reshape(-1, 2)
    pts = pts.astype(np.float32)
    # condition number of the level-0 template's G (integer points: the
    # bilinear samples are the stored integer gradients)
    rp = oracle.build_pyramid(I, 1)
    gx, gy = rp.gx[0].astype(np.int64), rp.gy[0].astype(np.int64)
    cond = []
    for px, py in pts.astype(int):
        wx, wy = gx[py - 10:py + 11, px - 10:px + 11], gy[py - 10:py + 11, px - 10:px + 11]
        a, b, c = int((wx * wx).sum()), int((wx * wy).sum()), int((wy * wy).sum())
        lmax = (a + c) / 2 + np.sqrt(((a - c) / 2) ** 2 + b * b)
        det = a * c - b * b
        cond.append(lmax * lmax / det if det > 0 else np.inf)
    cond = np.array(cond)
    ill = np.nonzero((cond > 1e5) & np.isfinite(cond))[0]
    prm = vt.KltParams(win=21, levels=levels, max_iters=30, eps=0.01, fb_thr=0.5, min_eig=1e-9)
    r0 = _ref(I, J, pts[ill], prm)
    r1 = _ref(I, J, pts[ill].astype(np.float64) + 1e-4, prm)
    moved = np.hypot(*(r0.pts - r1.pts).T)
    determined = (r0.status == r1.status) & ((r0.status == 0) | (moved <= 1e-3))
    sel = ill[determined]
    assert len(sel) >= 40 and determined.mean() >= 0.7, (len(ill), determined.mean())
    g = _gpu_track(I, J, pts[sel], prm)
    r = _ref(I, J, pts[sel], prm)
    st = compare(g["pts"], g["status"], g["reason"], r, f"cond > 1e5, theta {theta_deg}, period {lam}")
    print(f"ill-conditioned (theta {theta_deg}, period {lam}): {len(ill)} points with cond > 1e5 (median "
          f"{np.median(cond[ill]):.3g}), {len(ill) - len(sel)} undetermined by the data, {st}")
    assert st["tracked_ref"] >= 0.5 * len(sel), st
    # the batched launches take the same FP64 route: equal to the single-pair call
    import torch

    pI, pJ = vt.vt_pyramid_build_grad(I, levels), vt.vt_pyramid_build_grad(J, levels)
    p0 = torch.from_numpy(np.ascontiguousarray(pts[sel])).cuda()
    out, stt = torch.zeros((len(sel), 2), device="cuda"), torch.zeros(len(sel), dtype=torch.uint8, device="cuda")
    b = vt.Batch(1, 1)
    vt.vt_batch_set(b, [], [vt.track_task(pI, pJ, p0, out, stt, fb=False)], prm)
    vt.vt_batch_run(b)
    torch.cuda.synchronize()
    assert np.array_equal(stt.cpu().numpy(), g["status"])
    ok = g["status"] == 1
    assert np.array_equal(out.cpu().numpy()[ok], g["pts"][ok])
    b.free()
    pI.free()
    pJ.free()


@pytest.mark.parametrize("win", [9, 15, 21, 31])
def test_borders_and_tiny_levels_against_oracle(win):
    """Windows that cross every image edge, on a small smooth image with five
    levels (down to 4 x 3 px) and on a wider one with a window-wide margin:
    the staged template and footprint windows take their clamped-row chunk
    path, their one-column-per-lane path and (levels narrower than the
    window) only the latter.  Forward-backward tracking against the oracle
    under the usual flow and margin rules."""
    from scipy.ndimage import gaussian_filter

    vt = _vt()
    rng = np.random.Generator(np.random.PCG64(100 + win))
    for w, h in ((53, 37), (160, 96)):
        base = gaussian_filter(rng.uniform(0, 255, (h + 8, w + 8)), 1.5)
        I = np.clip(base[4:4 + h, 4:4 + w] * 1.6 - 70, 0, 255).astype(np.uint8)
        J = np.clip(base[3:3 + h, 6:6 + w] * 1.6 - 70, 0, 255).astype(np.uint8)  # (+2, +1) px shift
        xs = np.concatenate([[0, 0.5, 1.25, 3.0, w - 4.5, w - 2.0, w - 1.25, w - 1], rng.uniform(0, w - 1, 40)])
        ys = np.concatenate([[0, h - 1, 0.75, h - 2.5, 2.0, 3.5, h - 3.25, 0], rng.uniform(0, h - 1, 40)])
        pts = np.stack([xs, ys], 1).astype(np.float32)
        for levels in (1, 3, 5):
            prm = vt.KltParams(win=win, levels=levels, min_eig=1e-5)
            g = _gpu_track(I, J, pts, prm, fb=True)
            r = _ref(I, J, pts, prm, fb=True)
            st = _check(g, r, f"{w}x{h} win {win} L{levels}", fb=True)
            if levels < 5:  # at five levels the top is a few pixels wide: most points fail the eigenvalue test
                assert st["tracked_ref"] >= 30, st
