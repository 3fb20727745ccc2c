"""Batched persistent path (vt_batch_*): pyramids bit-exact against the
oracle, tracking equal to the single-pair calls and to the oracle, results
independent of the rest of the batch, CUDA-graph replay with new tables."""

import numpy as np
import pytest

import oracle
import synth
from parity import compare

pytestmark = pytest.mark.gpu


def _vt():
    import paper_2607_01757_gb300 as vt

    return vt


class Stream:
    """Device state of one synthetic camera stream for two consecutive frames."""

    def __init__(self, spec, frames, torch, vt, unaligned=False):
        self.spec = spec
        self.fr = frames
        L = spec.levels
        dev = "cuda"

        def up(a):
            t = torch.from_numpy(a).to(dev)
            if unaligned:  # odd pitch and an odd base offset -> byte staging path
                big = torch.zeros((a.shape[0], a.shape[1] + 3), dtype=torch.uint8, device=dev)
                big[:, 1:1 + a.shape[1]] = t
                return big[:, 1:1 + a.shape[1]]
            return t

        self.left = [up(a) for a in frames.left]
        self.right = [up(a) if a is not None else None for a in frames.right]
        self.kps = [torch.from_numpy(k).to(dev) for k in frames.kps]
        self.pyr = [vt.vt_pyramid_create(spec.w, spec.h, L) for _ in range(2)]
        self.pyr_r = vt.vt_pyramid_create(spec.w, spec.h, L) if spec.stereo else None
        def mk(n):
            return (torch.zeros((n, 2), device=dev), torch.zeros(n, dtype=torch.uint8, device=dev),
                    torch.zeros(n, device=dev), torch.zeros(n, dtype=torch.uint8, device=dev))

        self.out_t = mk(self.kps[0].shape[0])
        self.out_s = mk(self.kps[1].shape[0]) if spec.stereo else None


def _streams(n, seed, torch, vt, levels=(4, 5, 6), unaligned_every=0, kp=(40, 160)):
    specs = synth.make_stream_mix(n, seed=seed, kp_range=kp, levels=levels)
    out = []
    for i, sp in enumerate(specs):
        # smaller frames than the workload keep the oracle fast; shapes stay uneven
        sp.w, sp.h = [(203, 131), (320, 240), (377, 241), (160, 120), (256, 200), (97, 65)][i % 6]
        fr = synth.render_stream_frames(sp, 2)
        out.append(Stream(sp, fr, torch, vt, unaligned=bool(unaligned_every and i % unaligned_every == 0)))
    return out


def _stage(vt, streams, prm, with_frame0=True):
    frames, tasks = [], []
    for s in streams:
        if with_frame0:
            frames.append(vt.frame_job(s.left[0], s.pyr[0]))
        frames.append(vt.frame_job(s.left[1], s.pyr[1]))
        if s.spec.stereo:
            frames.append(vt.frame_job(s.right[1], s.pyr_r))
    for s in streams:
        o = s.out_t
        tasks.append(vt.track_task(s.pyr[0], s.pyr[1], s.kps[0], o[0], o[1], o[2], fb=True, reason=o[3]))
        if s.spec.stereo:
            o = s.out_s
            tasks.append(vt.track_task(s.pyr[1], s.pyr_r, s.kps[1], o[0], o[1], o[2], fb=True, reason=o[3]))
    return frames, tasks


def _prm(vt, levels):
    return vt.KltParams(win=21, levels=levels, max_iters=30, eps=0.01, fb_thr=0.5)


def test_batched_pyramids_bit_exact_and_tracking_matches():
    import torch

    vt = _vt()
    streams = _streams(7, 41, torch, vt, unaligned_every=3)
    Lmin = min(s.spec.levels for s in streams)
    prm = _prm(vt, Lmin)
    b = vt.Batch(32, 32)
    frames, tasks = _stage(vt, streams, prm)
    vt.vt_batch_set(b, frames, tasks, prm)
    vt.vt_batch_run(b)
    torch.cuda.synchronize()
    for s in streams:
        for pyr, img in [(s.pyr[0], s.fr.left[0]), (s.pyr[1], s.fr.left[1])] + \
                ([(s.pyr_r, s.fr.right[1])] if s.spec.stereo else []):
            ref = oracle.build_pyramid(img, s.spec.levels)
            for l in range(s.spec.levels):
                assert np.array_equal(pyr.level(l).cpu().numpy(), ref.levels[l])
                g = pyr.grad(l).cpu().numpy()
                assert np.array_equal(g[..., 0], ref.gx[l]) and np.array_equal(g[..., 1], ref.gy[l])
    # tracking: equal to the single-pair fused call and within parity of the oracle
    for s in streams:
        pairs = [(s.pyr[0], s.pyr[1], s.kps[0], s.out_t, s.fr.left[0], s.fr.left[1], s.fr.kps[0])]
        if s.spec.stereo:
            pairs.append((s.pyr[1], s.pyr_r, s.kps[1], s.out_s, s.fr.left[1], s.fr.right[1], s.fr.kps[1]))
        for pI, pJ, kp, o, I, J, kpn in pairs:
            n = kp.shape[0]
            out = torch.zeros((n, 2), device="cuda")
            st = torch.zeros(n, dtype=torch.uint8, device="cuda")
            vt.vt_klt_track_fb(pI, pJ, kp, prm, out, st)
            torch.cuda.synchronize()
            assert torch.equal(st, o[1])
            ok = st.bool()
            assert torch.equal(out[ok], o[0][ok])
            r = oracle.track_fb(oracle.build_pyramid(I, prm.levels), oracle.build_pyramid(J, prm.levels), kpn,
                                prm.win, prm.levels, prm.max_iters, prm.eps, prm.min_eig, prm.fb_thr)
            compare(o[0].cpu().numpy(), o[1].cpu().numpy(), o[3].cpu().numpy(), r, "batched")
    b.free()


def test_result_alone_equals_result_in_mix_and_graph_replay():
    import torch

    vt = _vt()
    streams = _streams(6, 43, torch, vt)
    Lmin = min(s.spec.levels for s in streams)
    prm = _prm(vt, Lmin)
    b = vt.Batch(32, 32)
    # whole mix, graph path (first call captures)
    frames, tasks = _stage(vt, streams, prm)
    vt.vt_batch_set(b, frames, tasks, prm)
    vt.vt_batch_run_graph(b)
    torch.cuda.synchronize()
    mix = [(s.out_t[0].clone(), s.out_t[1].clone()) for s in streams]
    for s in streams:
        for o in (s.out_t,) + ((s.out_s,) if s.spec.stereo else ()):
            o[0].zero_()
            o[1].zero_()
    # each stream alone, replaying the graphs with different tables each time
    for i, s in enumerate(streams):
        f1, t1 = _stage(vt, [s], prm)
        vt.vt_batch_set(b, f1, t1, prm)
        vt.vt_batch_run_graph(b)
        torch.cuda.synchronize()
        assert torch.equal(s.out_t[1], mix[i][1])
        ok = s.out_t[1].bool()
        assert torch.equal(s.out_t[0][ok], mix[i][0][ok])
    info = vt.vt_batch_info(b)
    assert info["klt_grid"] > 0 and info["launches_per_run"] >= 2
    b.free()


def test_batch_tasks_without_frames_and_empty_runs():
    import torch

    vt = _vt()
    streams = _streams(3, 47, torch, vt, levels=(4,))
    prm = _prm(vt, 4)
    b = vt.Batch(8, 8)
    frames, tasks = _stage(vt, streams, prm)
    vt.vt_batch_set(b, frames, [], prm)  # pyramids only
    vt.vt_batch_run(b)
    vt.vt_batch_set(b, [], tasks, prm)  # tracking only, on the pyramids built above
    vt.vt_batch_run(b)
    vt.vt_batch_set(b, [], [], prm)  # nothing at all
    vt.vt_batch_run_graph(b)
    torch.cuda.synchronize()
    s = streams[0]
    n = s.kps[0].shape[0]
    out = torch.zeros((n, 2), device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    vt.vt_klt_track_fb(s.pyr[0], s.pyr[1], s.kps[0], prm, out, st)
    torch.cuda.synchronize()
    assert torch.equal(st, s.out_t[1])
    b.free()


def test_one_level_pyramid_in_batch():
    import torch

    vt = _vt()
    img = synth.texture.quantize_u8(synth.BlobTexture(3, extent=(-20, -20, 120, 100)).eval_affine(
        100, 80, np.array([[1.0, 0, 0], [0, 1.0, 0]])))
    d = torch.from_numpy(img).cuda()
    p = vt.vt_pyramid_create(100, 80, 1)
    b = vt.Batch(2, 1)
    vt.vt_batch_set(b, [vt.frame_job(d, p)], [], _prm(vt, 1))
    vt.vt_batch_run(b)
    torch.cuda.synchronize()
    ref = oracle.build_pyramid(img, 1)
    assert np.array_equal(p.level(0).cpu().numpy(), img)
    assert np.array_equal(p.grad(0).cpu().numpy()[..., 0], ref.gx[0])
    b.free()


def test_batch_argument_errors():
    import torch

    vt = _vt()
    b = vt.Batch(2, 2)
    p = vt.vt_pyramid_create(64, 48, 3)
    img = torch.zeros((48, 64), dtype=torch.uint8, device="cuda")
    prm = _prm(vt, 3)
    with pytest.raises(vt.VTError):  # same pyramid built twice in one run
        vt.vt_batch_set(b, [vt.frame_job(img, p), vt.frame_job(img, p)], [], prm)
    with pytest.raises(vt.VTError):  # too many frames for the capacity
        vt.vt_batch_set(b, [vt.frame_job(img, p)] * 3, [], prm)
    with pytest.raises(vt.VTError):  # run before anything was staged
        vt.vt_batch_run(vt.Batch(1, 1))
    q = vt.vt_pyramid_create(64, 48, 2)
    pts = torch.zeros((4, 2), device="cuda")
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(vt.VTError):  # levels beyond the target pyramid
        vt.vt_batch_set(b, [vt.frame_job(img, p), vt.frame_job(img, q)],
                        [vt.track_task(p, q, pts, pts, st)], prm)
    b.free()


@pytest.mark.parametrize("grad", [1, 2])
def test_batched_pyramids_at_workload_sizes(grad):
    """Tiled launches for the large levels and the tail kernel for the small
    ones: bit-exact at every stream shape of the workload, 1 to 6 levels."""
    import torch

    vt = _vt()
    shapes = [(640, 480, 4), (752, 480, 5), (960, 600, 6), (1440, 1080, 5), (1920, 1200, 6), (752, 480, 1),
              (97, 65, 3), (1920, 1200, 2)]
    rng = np.random.Generator(np.random.PCG64(5))
    frames, keep = [], []
    for i, (w, h, L) in enumerate(shapes):
        tex = synth.BlobTexture(50 + i, extent=(-40, -40, w + 40, h + 40), n_blobs=int(400 * w * h / 361000),
                                blob_radius_sigmas=4.0)
        img = synth.texture.quantize_u8(tex.eval_affine(w, h, np.array([[1.0, 0, 0], [0, 1.0, 0]])))
        img.reshape(-1)[rng.integers(0, w * h, 16)] = 255
        d = torch.from_numpy(img).cuda()
        p = vt.vt_pyramid_create(w, h, L)
        frames.append(vt.frame_job(d, p))
        keep.append((img, d, p, L))
    b = vt.Batch(len(frames), 1)
    vt.vt_batch_set(b, frames, [], vt.KltParams(levels=1), grad_type=grad)
    vt.vt_batch_run_graph(b)
    torch.cuda.synchronize()
    for img, d, p, L in keep:
        ref = oracle.build_pyramid(img, L)
        for l in range(L):
            assert np.array_equal(p.level(l).cpu().numpy(), ref.levels[l]), (img.shape, L, l)
            g = p.grad(l).cpu().numpy()
            if grad == 1:
                assert np.array_equal(g[..., 0], ref.gx[l]) and np.array_equal(g[..., 1], ref.gy[l]), (img.shape, l)
            else:
                ex = (ref.gx[l] / 32.0).astype(np.float16)
                assert np.array_equal(g[..., 0].view(np.uint16), ex.view(np.uint16)), (img.shape, l)
    b.free()


def test_levels_timed_run_and_fma_probe():
    """vt_batch_run_levels_timed records an event after every pyramid launch
    of the staged run (and refuses too few events); the FP32 FMA probe
    returns its FLOP count and runs at a plausible rate."""
    import torch

    vt = _vt()
    streams = _streams(3, 51, torch, vt)
    prm = _prm(vt, min(s.spec.levels for s in streams))
    b = vt.Batch(32, 32)
    frames, tasks = _stage(vt, streams, prm)
    vt.vt_batch_set(b, frames, tasks, prm)
    n_pyr = vt.vt_batch_info(b)["launches_per_run"] - 1
    ev = []
    for _ in range(4 + n_pyr):
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        ev.append(e)
    with pytest.raises(vt.VTError):
        vt.vt_batch_run_levels_timed(b, None, ev[:3 + n_pyr])
    vt.vt_batch_run_levels_timed(b, None, ev)
    torch.cuda.synchronize()
    ms = [ev[0].elapsed_time(ev[4])] + [ev[4 + j - 1].elapsed_time(ev[4 + j]) for j in range(1, n_pyr)]
    assert all(m >= 0 for m in ms) and ev[0].elapsed_time(ev[1]) >= sum(ms) * 0.999
    b.free()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(sms * 2048, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fl = vt.vt_fp32_fma_probe(512, out)
    e1.record()
    torch.cuda.synchronize()
    assert fl == sms * 8 * 256 * 8 * 8 * 512 * 2
    tflops = fl / (e0.elapsed_time(e1) / 1e3) / 1e12
    assert 5.0 < tflops < 200.0, tflops
    assert torch.isfinite(out).all()
    with pytest.raises(vt.VTError):
        vt.vt_fp32_fma_probe(512, out[:100])
