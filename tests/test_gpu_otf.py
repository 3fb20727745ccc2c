"""Gradients computed inside the tracker (pyramids without Scharr planes,
VT_GRAD_NONE) against stored int16 gradients: the tracker recomputes the
same integers, so every output must be bit-identical -- on the workloads,
near every border, on tiny coarse levels, for every supported window, with
and without an initial guess, alone and in a batched run -- and therefore
within the parity rule of the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


def _track(vt, I, J, pts, prm, grad, fb=True, guess=None):
    import torch

    build = (lambda img: vt.vt_pyramid_build(img, prm.levels)) if grad == vt.VT_GRAD_NONE else \
        (lambda img: vt.vt_pyramid_build_grad(img, prm.levels, grad))
    pI, pJ = build(I), build(J)
    n = len(pts)
    p0 = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    out = torch.zeros((n, 2), device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    err = torch.zeros(n, device="cuda")
    rs = torch.zeros(n, dtype=torch.uint8, device="cuda")
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    if fb:
        vt.vt_klt_track_fb(pI, pJ, p0, prm, out, st, err, reason=rs, iters=it)
    else:
        g = None if guess is None else torch.from_numpy(np.ascontiguousarray(guess, np.float32)).cuda()
        vt.vt_klt_track_ex(pI, pJ, p0, prm, out, st, err, pts_guess=g, reason=rs, iters=it)
    torch.cuda.synchronize()
    res = [t.cpu().numpy() for t in (out, st, err, rs, it)]
    pI.free()
    pJ.free()
    return res


def _equal(a, b, label):
    for k, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), (label, k)


def test_otf_bit_identical_on_workloads():
    import paper_2607_01757_gb300 as vt

    c = synth.make_config1(1)
    prm = vt.KltParams(win=21, levels=4)
    a = _track(vt, c.I, c.J, c.pts, prm, vt.VT_GRAD_NONE)
    _equal(a, _track(vt, c.I, c.J, c.pts, prm, vt.VT_GRAD_S16), "config 1")
    r = oracle.track_fb(oracle.build_pyramid(c.I, 4), oracle.build_pyramid(c.J, 4), c.pts, 21, 4, 30, 0.01, 1e-4,
                        0.5)
    compare(a[0], a[1], a[3], r, "otf config 1")
    seq = synth.make_stereo_sequence(seed=2, n_frames=2, w=752, h=480, n_kp=1000)
    prm = vt.KltParams(win=21, levels=5)
    for I, J, pts in [(seq.left[0], seq.left[1], seq.kps[0]), (seq.left[1], seq.right[1], seq.kps[1])]:
        _equal(_track(vt, I, J, pts, prm, vt.VT_GRAD_NONE), _track(vt, I, J, pts, prm, vt.VT_GRAD_S16), "sequence")


@pytest.mark.parametrize("win", [9, 15, 21, 31])
def test_otf_bit_identical_at_borders_and_tiny_levels(win):
    """A 45 x 23 image with 5 levels (down to 3 x 2 px): every window reaches
    the reflected first / last rows and columns; points on and near every
    edge, plus a guessed start."""
    import paper_2607_01757_gb300 as vt

    rng = np.random.Generator(np.random.PCG64(win))
    w, h = 45, 23
    I = rng.integers(0, 256, (h, w), dtype=np.uint8)
    J = np.roll(I, (1, -2), axis=(0, 1))
    xs = np.concatenate([[0, 0.4, 1, 2.5, w - 3.5, w - 2, w - 1.2, w - 1], rng.uniform(0, w - 1, 24)])
    ys = np.concatenate([[0, h - 1, 0.7, h - 1.5, 1, 2.2, h - 2.6, 0], rng.uniform(0, h - 1, 24)])
    pts = np.stack([xs, ys], 1).astype(np.float32)
    for levels in (1, 3, 5):
        prm = vt.KltParams(win=win, levels=levels, min_eig=1e-6)
        _equal(_track(vt, I, J, pts, prm, vt.VT_GRAD_NONE), _track(vt, I, J, pts, prm, vt.VT_GRAD_S16),
               f"fb L{levels}")
        guess = pts + np.float32([-2.0, 1.0])
        _equal(_track(vt, I, J, pts, prm, vt.VT_GRAD_NONE, fb=False, guess=guess),
               _track(vt, I, J, pts, prm, vt.VT_GRAD_S16, fb=False, guess=guess), f"guess L{levels}")
    # one-row and one-column images
    for shape in ((1, 40), (40, 1), (2, 3)):
        I1 = rng.integers(0, 256, shape, dtype=np.uint8)
        p1 = np.array([[0.0, 0.0], [shape[1] - 1, shape[0] - 1]], np.float32)
        prm = vt.KltParams(win=win, levels=2, min_eig=0.0)
        _equal(_track(vt, I1, I1, p1, prm, vt.VT_GRAD_NONE, fb=False),
               _track(vt, I1, I1, p1, prm, vt.VT_GRAD_S16, fb=False), f"{shape}")


def test_otf_batched_bit_identical():
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.engine import BatchedTracker

    specs = synth.make_stream_mix(10, seed=8)
    pick = [sp for sp in specs if sp.w <= 960][:4]
    frames = [synth.render_stream_frames(sp, 2) for sp in pick]
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    outs = []
    for grad in (vt.VT_GRAD_NONE, vt.VT_GRAD_S16):
        tr = BatchedTracker(pick, vt.KltParams(), grad_type=grad)
        sids = list(range(len(pick)))
        tr.stage(tr.step_tables(sids, [0] * len(sids), [0] * len(sids), [dev(f.left[0]) for f in frames],
                                [dev(f.right[0]) for f in frames]))
        tr.run(graph=False)
        tr.advance(sids)
        tr.stage(tr.step_tables(sids, [len(f.kps[0]) for f in frames], [len(f.kps[1]) for f in frames],
                                [dev(f.left[1]) for f in frames], [dev(f.right[1]) for f in frames],
                                kpt=[dev(f.kps[0]) for f in frames], kps=[dev(f.kps[1]) for f in frames]))
        tr.run(graph=True)
        torch.cuda.synchronize()
        o = []
        for s in tr.streams:
            o += [t.cpu().numpy() for t in s.out_t]
            if s.stereo:
                o += [t.cpu().numpy() for t in s.out_s]
        outs.append(o)
        tr.free()
    _equal(outs[0], outs[1], "batched")
