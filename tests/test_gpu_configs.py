"""Parity at the workload configurations, through the C ABI:

* stereo + temporal sequence, 752x480, 1000 keypoints (NMS radius 4), 5 levels:
  prev->cur and left->right, each forward-backward checked;
* the precision workload, 1280x1024, 2000 keypoints, motion blur and exposure
  change: full parity with int16 gradients, and the error of the FP16-gradient
  variant against the FP64 oracle (on int16 gradients) stated and bounded;
* full-size stream shapes through the batched launch the benchmark times, on
  a sample of points the oracle tracks one by one.
"""

import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


def _gpu_fb(I, J, pts, prm, grad):
    import torch

    import paper_2607_01757_gb300 as vt

    pI = vt.vt_pyramid_build_grad(I, prm.levels, grad)
    pJ = vt.vt_pyramid_build_grad(J, prm.levels, grad)
    n = len(pts)
    p0 = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    out = torch.zeros((n, 2), device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    err = torch.zeros(n, device="cuda")
    rs = torch.zeros(n, dtype=torch.uint8, device="cuda")
    vt.vt_klt_track_fb(pI, pJ, p0, prm, out, st, err, reason=rs)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), st.cpu().numpy(), err.cpu().numpy(), rs.cpu().numpy()
    pI.free()
    pJ.free()
    return res


def _oracle_fb(I, J, pts, prm):
    return oracle.track_fb(oracle.build_pyramid(I, prm.levels), oracle.build_pyramid(J, prm.levels), pts, prm.win,
                           prm.levels, prm.max_iters, prm.eps, prm.min_eig, prm.fb_thr)


def test_stereo_temporal_sequence_752x480():
    import paper_2607_01757_gb300 as vt

    seq = synth.make_stereo_sequence(seed=2, n_frames=2, w=752, h=480, n_kp=1000)
    prm = vt.KltParams(win=21, levels=5, max_iters=30, eps=0.01, fb_thr=0.5)
    for I, J, pts, label in [(seq.left[0], seq.left[1], seq.kps[0], "temporal"),
                             (seq.left[1], seq.right[1], seq.kps[1], "stereo")]:
        assert len(pts) == 1000
        g_pts, g_st, g_err, g_rs = _gpu_fb(I, J, pts, prm, vt.VT_GRAD_S16)
        r = _oracle_fb(I, J, pts, prm)
        st = compare(g_pts, g_st, g_rs, r, label)
        assert st["tracked_ref"] > 500, st


@pytest.fixture(scope="module")
def precision_seq():
    return synth.make_config3_pair(seed=3)


def test_precision_workload_1280x1024_int16(precision_seq):
    import paper_2607_01757_gb300 as vt

    seq = precision_seq
    prm = vt.KltParams(win=21, levels=5, max_iters=30, eps=0.01, fb_thr=0.5)
    I, J, pts = seq.left[0], seq.left[1], seq.kps[0]
    assert len(pts) == 2000
    g_pts, g_st, _, g_rs = _gpu_fb(I, J, pts, prm, vt.VT_GRAD_S16)
    r = _oracle_fb(I, J, pts, prm)
    compare(g_pts, g_st, g_rs, r, "1280x1024 int16")


def test_precision_workload_fp16_gradients_error_stated(precision_seq):
    """FP16 gradient storage changes the weights of b = sum r grad T and the
    eigenvalue test by the half-precision rounding of raw/32 (relative
    2^-11) wherever an odd Scharr response exceeds 2048 (smaller or even
    responses are exact in half precision), so its flow may differ from the
    FP64 oracle on int16 gradients by a small amount and a few eigenvalue
    decisions near the threshold may flip.  Measured and bounded here."""
    import paper_2607_01757_gb300 as vt

    seq = precision_seq
    prm = vt.KltParams(win=21, levels=5, max_iters=30, eps=0.01, fb_thr=0.5)
    I, J, pts = seq.left[0], seq.left[1], seq.kps[0]
    g_pts, g_st, _, _ = _gpu_fb(I, J, pts, prm, vt.VT_GRAD_F16)
    r = _oracle_fb(I, J, pts, prm)
    both = (g_st == 1) & (r.status == 1)
    d = np.hypot(*(g_pts[both] - r.fwd.pts[both]).T)
    stats = dict(mean=float(d.mean()), p99=float(np.percentile(d, 99)), max=float(d.max()),
                 status_agree=float((g_st == r.status).mean()), tracked=int(both.sum()))
    print("fp16 gradients vs fp64 oracle:", stats)
    assert stats["status_agree"] >= 0.99, stats
    assert stats["mean"] < 0.005 and stats["p99"] < 0.02 and stats["max"] < 0.05, stats


def half_rounded_fraction(pyr, pts, win=21, levels=1):
    """Fraction of the gradient components in the (win + 1)^2 footprints of
    the points' level-l templates (l < levels) whose half-precision storage
    of raw/32 is inexact: an odd raw Scharr response above 2048 in
    magnitude (half precision keeps 11 significant bits)."""
    hw = win // 2
    tot = rnd = 0
    for l in range(levels):
        gx, gy = pyr.gx[l].astype(np.int32), pyr.gy[l].astype(np.int32)
        bad = ((np.abs(gx) > 2048) & (gx % 2 != 0)).astype(np.int32) + \
            ((np.abs(gy) > 2048) & (gy % 2 != 0)).astype(np.int32)
        h, w = gx.shape
        for x, y in np.asarray(pts, np.float64) / 2 ** l:
            x0, y0 = int(np.floor(x)) - hw, int(np.floor(y)) - hw
            ys = np.clip(np.arange(y0, y0 + win + 1), 0, h - 1)
            xs = np.clip(np.arange(x0, x0 + win + 1), 0, w - 1)
            rnd += int(bad[np.ix_(ys, xs)].sum())
            tot += 2 * len(ys) * len(xs)
    return rnd / tot


def test_precision_high_contrast_fp16_error_exercised():
    """The precision configuration on a high-contrast variant (1280x1024,
    2000 keypoints, unblurred step edges, exposure x1.3 on the second frame),
    where odd Scharr responses above 2048 occur inside the windows, so FP16
    gradient storage does round.  int16 storage meets full parity with the
    FP64 oracle; FP16 storage's error against the oracle is stated (mean,
    p99, max px, fraction of window samples rounded) and bounded, and it is
    not zero: FP16 flows differ from int16 flows."""
    import paper_2607_01757_gb300 as vt

    c = synth.make_config3_contrast_pair(seed=5)
    prm = vt.KltParams(win=21, levels=5, max_iters=30, eps=0.01, fb_thr=0.5)
    r = _oracle_fb(c.I, c.J, c.pts, prm)
    s_pts, s_st, _, s_rs = _gpu_fb(c.I, c.J, c.pts, prm, vt.VT_GRAD_S16)
    st16 = compare(s_pts, s_st, s_rs, r, "high-contrast int16")
    h_pts, h_st, _, _ = _gpu_fb(c.I, c.J, c.pts, prm, vt.VT_GRAD_F16)
    both = (h_st == 1) & (r.status == 1)
    d = np.hypot(*(h_pts[both] - r.fwd.pts[both]).T)
    frac = half_rounded_fraction(oracle.build_pyramid(c.I, 5), c.pts, 21, 5)
    stats = dict(mean=float(d.mean()), p99=float(np.percentile(d, 99)), max=float(d.max()),
                 status_agree=float((h_st == r.status).mean()), tracked=int(both.sum()),
                 rounded_samples=frac, int16=st16)
    print("high-contrast fp16 gradients vs fp64 oracle:", stats)
    assert frac > 1e-3, stats
    changed = (h_st == 1) & (s_st == 1) & np.any(h_pts != s_pts, axis=1)
    assert changed.sum() > 0, "FP16 storage changed no flow"
    assert stats["status_agree"] >= 0.99, stats
    # reported, not bound by the 0.01 px rule (the precision configuration
    # states its error); measured mean 1.3e-4, p99 2.2e-4, max 0.088 px
    assert stats["mean"] < 0.002 and stats["p99"] < 0.01 and stats["max"] < 0.25, stats


@pytest.mark.parametrize("warps", [4, 8])
def test_full_size_streams_batched_sampled(warps):
    """The batched launch of the benchmark on full-size stream shapes (one
    stream of each shape, stereo and mono), every point tracked on the GPU,
    a sample of 48 points per task re-tracked by the oracle one by one; with
    either launch shape the benchmark's tuner can pick (4 or 8 warps per CTA)."""
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.engine import BatchedTracker

    specs = synth.make_stream_mix(32, seed=4)
    pick = []
    for shape in synth.scenes.STREAM_SHAPES:
        cand = [sp for sp in specs if (sp.w, sp.h) == shape]
        if cand:
            pick.append(cand[0])
    frames = [synth.render_stream_frames(sp, 2) for sp in pick]
    prm = vt.KltParams()
    tr = BatchedTracker(pick, prm)
    vt.vt_batch_config(tr.batch, warps, 0, 0)
    sids = list(range(len(pick)))
    L0 = [torch.from_numpy(f.left[0]).cuda() for f in frames]
    L1 = [torch.from_numpy(f.left[1]).cuda() for f in frames]
    R0 = [torch.from_numpy(f.right[0]).cuda() if f.right[0] is not None else None for f in frames]
    R1 = [torch.from_numpy(f.right[1]).cuda() if f.right[1] is not None else None for f in frames]
    k0 = [torch.from_numpy(f.kps[0]).cuda() for f in frames]
    k1 = [torch.from_numpy(f.kps[1]).cuda() for f in frames]
    n0 = [len(f.kps[0]) for f in frames]
    n1 = [len(f.kps[1]) for f in frames]
    tr.stage(tr.step_tables(sids, [0] * len(sids), [0] * len(sids), L0, R0))
    tr.run(graph=False)
    tr.advance(sids)
    tr.stage(tr.step_tables(sids, n0, n1, L1, R1, kpt=k0, kps=k1))
    tr.run(graph=True)
    tr.advance(sids)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(17))
    for i, (sp, f) in enumerate(zip(pick, frames)):
        s = tr.streams[i]
        prm_s = vt.KltParams(levels=sp.levels)
        tasks = [(f.left[0], f.left[1], f.kps[0], s.out_t)]
        if sp.stereo:
            tasks.append((f.left[1], f.right[1], f.kps[1], s.out_s))
        for I, J, kp, out in tasks:
            idx = np.sort(rng.choice(len(kp), size=min(48, len(kp)), replace=False))
            r = _oracle_fb(I, J, kp[idx], prm_s)
            compare(out[0].cpu().numpy(), out[1].cpu().numpy(), out[3].cpu().numpy(), r, f"{sp.w}x{sp.h} L{sp.levels}",
                    idx=idx)
    tr.free()


def test_stereo_temporal_sequence_six_frames_batched():
    """The stereo + temporal sequence stepped frame by frame through the
    batched engine (one stereo stream, 752x480, 1000 keypoints per frame,
    5 levels): at every step prev->cur and left->right tracking of a sample
    of 120 points agree with the oracle."""
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.engine import BatchedTracker

    F = 6
    seq = synth.make_stereo_sequence(seed=2, n_frames=F, w=752, h=480, n_kp=1000)
    spec = synth.StreamSpec(sid=0, w=752, h=480, stereo=True, n_kp=1000, levels=5, seed=2)
    tr = BatchedTracker([spec], vt.KltParams(win=21, levels=5))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    rng = np.random.Generator(np.random.PCG64(31))
    for t in range(F):
        L, R = dev(seq.left[t]), dev(seq.right[t])
        n_t = len(seq.kps[t - 1]) if t > 0 else 0
        kt = dev(seq.kps[t - 1]) if t > 0 else dev(seq.kps[0])
        tr.stage(tr.step_tables([0], [n_t], [len(seq.kps[t])], [L], [R], kpt=[kt], kps=[dev(seq.kps[t])]))
        tr.run(graph=True)
        tr.advance([0])
        torch.cuda.synchronize()
        s = tr.streams[0]
        tasks = [(seq.left[t], seq.right[t], seq.kps[t], s.out_s, "stereo")]
        if t > 0:
            tasks.append((seq.left[t - 1], seq.left[t], seq.kps[t - 1], s.out_t, "temporal"))
        for I, J, kp, out, label in tasks:
            idx = np.sort(rng.choice(len(kp), size=120, replace=False))
            r = _oracle_fb(I, J, kp[idx], vt.KltParams(win=21, levels=5))
            compare(out[0].cpu().numpy(), out[1].cpu().numpy(), out[3].cpu().numpy(), r, f"frame {t} {label}",
                    idx=idx)
    tr.free()


def test_stereo_temporal_sequence_64_frames_pool_aging_batched():
    """The stereo + temporal configuration as specified: 64 frames per
    camera at 752x480 (camera rotation up to 5 degrees per frame, 0.3 m/s at
    20 Hz), 1000 keypoints per frame, 5 levels, stepped frame by frame
    through the batched engine.  The temporal task tracks a pool that ages:
    the survivors of the previous step's forward-backward check keep being
    tracked from their GPU positions, topped up with the previous frame's
    new keypoints to 1000; the stereo task checks the current frame's
    keypoints left->right.  At every frame both tasks agree with the oracle
    on a seeded sample of 60 points each (the oracle tracks the same inputs)."""
    import multiprocessing as mp
    import os

    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.engine import BatchedTracker

    F, N = 64, 1000
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        seq = synth.make_stereo_sequence(seed=2, n_frames=F, w=752, h=480, n_kp=N, map_fn=pool.map)
    spec = synth.StreamSpec(sid=0, w=752, h=480, stereo=True, n_kp=N, levels=5, seed=2)
    prm = vt.KltParams(win=21, levels=5)
    tr = BatchedTracker([spec], prm)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=a.dtype)).cuda()  # noqa: E731
    rng = np.random.Generator(np.random.PCG64(64))
    pool_pts = seq.kps[0].copy()
    age = np.zeros(len(pool_pts), np.int64)
    max_age, checked = 0, 0
    for t in range(F):
        L, R = dev(seq.left[t]), dev(seq.right[t])
        n_t = len(pool_pts) if t > 0 else 0
        kt = dev(pool_pts.astype(np.float32))
        tr.stage(tr.step_tables([0], [n_t], [N], [L], [R], kpt=[kt], kps=[dev(seq.kps[t])]))
        tr.run(graph=True)
        tr.advance([0])
        torch.cuda.synchronize()
        s = tr.streams[0]
        tasks = [(seq.left[t], seq.right[t], seq.kps[t], s.out_s, "stereo")]
        if t > 0:
            tasks.append((seq.left[t - 1], seq.left[t], pool_pts, s.out_t, "temporal"))
        for I, J, kp, out, label in tasks:
            n = len(kp)
            idx = np.sort(rng.choice(n, size=60, replace=False))
            r = _oracle_fb(I, J, kp[idx].astype(np.float32), prm)
            compare(out[0][:n].cpu().numpy(), out[1][:n].cpu().numpy(), out[3][:n].cpu().numpy(), r,
                    f"frame {t} {label}", idx=idx)
            checked += 1
        if t > 0:
            ok = s.out_t[1][:n_t].cpu().numpy() == 1
            surv = s.out_t[0][:n_t].cpu().numpy()[ok]
            age = age[ok] + 1
            fresh = seq.kps[t][:N - len(surv)]
            pool_pts = np.concatenate([surv, fresh]).astype(np.float32)
            age = np.concatenate([age, np.zeros(len(fresh), np.int64)])
            max_age = max(max_age, int(age.max()))
    tr.free()
    assert checked == 2 * F - 1
    assert max_age >= 20, max_age  # some tracks live through a third of the sequence


@pytest.mark.parametrize("grad", ["s16", "f16", "none"])
def test_input_ring_equals_input_slots(grad):
    """A tracker over an input ring (each slot level 0 of its own pyramid,
    frames never copied) gives bit-identical points, status and errors to the
    tracker that copies each frame from its input slot, batched and plain,
    with int16, half or no stored gradient planes."""
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.engine import BatchedTracker

    specs = synth.make_stream_mix(16, seed=9, kp_range=(150, 400))
    pick = [sp for sp in specs if sp.stereo][:2] + [sp for sp in specs if not sp.stereo][:1]
    F = 3
    frames = [synth.render_stream_frames(sp, F) for sp in pick]

    def slot(img):
        h, w = img.shape
        p = (w + 15) // 16 * 16
        buf = torch.zeros(p * h + 64, dtype=torch.uint8, device="cuda")
        v = buf[:p * h].view(h, p)[:, :w]
        v.copy_(torch.from_numpy(img))
        return v

    ring = [([slot(f.left[k]) for k in range(F)], [slot(f.right[k]) for k in range(F)] if sp.stereo else None)
            for sp, f in zip(pick, frames)]
    prm = vt.KltParams()
    gt = {"s16": vt.VT_GRAD_S16, "f16": vt.VT_GRAD_F16, "none": vt.VT_GRAD_NONE}[grad]
    tr_r = BatchedTracker(pick, prm, grad_type=gt, ring=ring)
    tr_s = BatchedTracker(pick, prm, grad_type=gt)
    sids = list(range(len(pick)))
    dev = lambda a: torch.from_numpy(a).cuda() if a is not None else None  # noqa: E731
    kp = [[dev(f.kps[k]) for k in range(F)] for f in frames]
    for plain in (False, True):
        for t in range(F):
            n_t = [len(f.kps[t - 1]) if t > 0 else 0 for f in frames]
            n_s = [len(f.kps[t]) for f in frames]
            kt = [kp[i][t - 1] if t > 0 else kp[i][0] for i in sids]
            ks = [kp[i][t] for i in sids]
            L = [dev(f.left[t]) for f in frames]
            R = [dev(f.right[t]) for f in frames]
            ri = [((t - 1) % F, t)] * len(sids)
            if plain:
                tr_r.plain_step(sids, n_t, n_s, kpt=kt, kps=ks, ring_idx=ri)
                tr_s.plain_step(sids, n_t, n_s, L, R, kpt=kt, kps=ks)
            else:
                tr_r.stage(tr_r.step_tables(sids, n_t, n_s, kpt=kt, kps=ks, ring_idx=ri))
                tr_r.run(graph=True)
                tr_s.stage(tr_s.step_tables(sids, n_t, n_s, L, R, kpt=kt, kps=ks))
                tr_s.run(graph=True)
            tr_r.advance(sids)
            tr_s.advance(sids)
            torch.cuda.synchronize()
            for a, b in ((tr_r.out_pts, tr_s.out_pts), (tr_r.out_st, tr_s.out_st), (tr_r.out_err, tr_s.out_err)):
                assert torch.equal(a, b), (plain, t)
            assert int(tr_r.out_st.sum().item()) > 0
    with pytest.raises(ValueError):  # a ring stream's step names its slots
        tr_r.step_tables(sids, [0] * 3, [0] * 3)
    tr_r.free()
    tr_s.free()
