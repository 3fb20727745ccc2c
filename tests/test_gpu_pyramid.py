"""Pyramid (K1) and Scharr gradients (K2): bit-exact against the oracle,
through the C ABI, on tiny, ragged and full-size images."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (2, 3), (5, 1), (1, 7), (7, 7), (8, 8), (17, 33), (63, 65), (129, 47), (200, 131), (752, 480),
         (640, 480), (1280, 1024), (1920, 1200)]


def _img(w, h, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    if w * h < 4096:
        return rng.integers(0, 256, (h, w), dtype=np.uint8)
    tex = synth.BlobTexture(seed, extent=(-50, -50, w + 50, h + 50), n_blobs=max(20, int(400 * w * h / 361000)),
                            blob_radius_sigmas=4.0)
    img = synth.texture.quantize_u8(tex.eval_affine(w, h, np.array([[1.0, 0, 0], [0, 1.0, 0]])))
    # salt a few extreme pixels so saturating values are exercised
    idx = rng.integers(0, w * h, 64)
    img.reshape(-1)[idx[:32]] = 0
    img.reshape(-1)[idx[32:]] = 255
    return img


def _levels_for(w, h):
    return max(1, min(6, int(np.log2(max(1, min(w, h)))) + 2))


@pytest.mark.parametrize("w,h", SIZES)
def test_pyramid_and_gradients_bit_exact(w, h):
    import torch

    import paper_2607_01757_gb300 as vt

    img = _img(w, h, seed=w * 1000 + h)
    L = _levels_for(w, h)
    ref = oracle.build_pyramid(img, L)
    # device input, separate gradient pass
    dimg = torch.from_numpy(img).cuda()
    p = vt.vt_pyramid_build(dimg, L)
    vt.vt_gradients(p, vt.VT_GRAD_S16)
    # host input, fused pyramid + gradients
    q = vt.vt_pyramid_build_grad(img, L, vt.VT_GRAD_S16)
    torch.cuda.synchronize()
    for l in range(L):
        for pyr in (p, q):
            lv = pyr.level(l).cpu().numpy()
            assert lv.shape == ref.levels[l].shape
            assert np.array_equal(lv, ref.levels[l]), (w, h, l)
            g = pyr.grad(l).cpu().numpy()
            assert np.array_equal(g[..., 0], ref.gx[l]), (w, h, l)
            assert np.array_equal(g[..., 1], ref.gy[l]), (w, h, l)
    p.free()
    q.free()


@pytest.mark.parametrize("w,h", [(7, 5), (752, 480), (1280, 1024)])
def test_f16_gradients_round_to_nearest_even(w, h):
    import torch

    import paper_2607_01757_gb300 as vt

    img = _img(w, h, seed=7 * w + h)
    L = _levels_for(w, h)
    ref = oracle.build_pyramid(img, L)
    p = vt.vt_pyramid_build_grad(img, L, vt.VT_GRAD_F16)
    q = vt.vt_pyramid_build(img, L)
    vt.vt_gradients(q, vt.VT_GRAD_F16)
    torch.cuda.synchronize()
    for l in range(L):
        # numpy's float64 -> float16 conversion rounds to nearest even
        ex = (ref.gx[l] / 32.0).astype(np.float16)
        ey = (ref.gy[l] / 32.0).astype(np.float16)
        for pyr in (p, q):
            g = pyr.grad(l).cpu().numpy()
            assert np.array_equal(g[..., 0].view(np.uint16), ex.view(np.uint16))
            assert np.array_equal(g[..., 1].view(np.uint16), ey.view(np.uint16))


def test_rebuild_in_place_and_pitch():
    import torch

    import paper_2607_01757_gb300 as vt

    a = _img(300, 200, 1)
    b = _img(300, 200, 2)
    p = vt.vt_pyramid_build_grad(a, 4, vt.VT_GRAD_S16)
    h0 = p.handle
    # a strided device view of a wider buffer as input (pitch > width)
    big = torch.zeros((200, 320), dtype=torch.uint8, device="cuda")
    big[:, :300] = torch.from_numpy(b).cuda()
    vt.vt_pyramid_build_grad(big[:, :300], 4, vt.VT_GRAD_S16, out=p)
    torch.cuda.synchronize()
    assert p.handle == h0
    ref = oracle.build_pyramid(b, 4)
    for l in range(4):
        assert np.array_equal(p.level(l).cpu().numpy(), ref.levels[l])
        assert np.array_equal(p.grad(l).cpu().numpy()[..., 0], ref.gx[l])
    # a mismatched shape is refused
    with pytest.raises(vt.VTError):
        vt.vt_pyramid_build_grad(_img(301, 200, 3), 4, vt.VT_GRAD_S16, out=p)
    w, h, L, nbytes = p.info()
    assert (w, h, L) == (300, 200, 4) and nbytes > 0


@pytest.mark.parametrize("w,h", [(752, 480), (1440, 1080), (97, 65)])
def test_frame_uploaded_into_level0_builds_in_place(w, h):
    """A frame copied into the pyramid's own level 0 (vt_pyramid_upload) and
    built with level 0 named as its image gives the same pyramid and
    gradients as a build from a separate image, through the single-pair call
    and through the batched launches; level 0 keeps the frame.  Naming level
    0 with another pitch is an argument error."""
    import torch

    import paper_2607_01757_gb300 as vt

    img = _img(w, h, seed=7 * w + h)
    L = _levels_for(w, h)
    ref = oracle.build_pyramid(img, L)
    a = vt.vt_pyramid_create(w, h, L)
    vt.vt_pyramid_upload(a, img)
    vt.vt_pyramid_build_grad(a.level(0), L, vt.VT_GRAD_S16, out=a)
    b = vt.vt_pyramid_create(w, h, L)
    vt.vt_pyramid_upload(b, torch.from_numpy(img).cuda())
    batch = vt.Batch(2, 1)
    vt.vt_batch_set(batch, [vt.frame_job(b.level(0), b)], [], vt.KltParams(levels=L))
    vt.vt_batch_run(batch)
    torch.cuda.synchronize()
    for p in (a, b):
        for l in range(L):
            assert np.array_equal(p.level(l).cpu().numpy(), ref.levels[l]), l
            g = p.grad(l).cpu().numpy()
            assert np.array_equal(g[..., 0], ref.gx[l]) and np.array_equal(g[..., 1], ref.gy[l]), l
    lv0 = b.level(0)
    if lv0.stride(0) != w:  # a view of b's level 0 with another pitch
        bad = torch.as_strided(lv0, (h, w - 1), (lv0.stride(0) - 1, 1)) if h > 1 else None
        if bad is not None:
            with pytest.raises(vt.VTError):
                vt.vt_batch_set(batch, [vt.frame_job(bad, b)], [], vt.KltParams(levels=L))
    batch.free()
    a.free()
    b.free()


@pytest.mark.parametrize("w,h", [(752, 480), (1440, 1080), (97, 65), (16, 3)])
def test_pyramid_on_caller_level0(w, h):
    """A pyramid whose level 0 is the caller's buffer (vt_pyramid_create_on):
    built in place by the single-pair call and by the batched launches, it
    equals the oracle bit for bit, level 0 stays the caller's frame, tracking
    against it gives the owned pyramid's results, the buffer outlives the
    pyramid, and bad layouts are argument errors."""
    import torch

    import paper_2607_01757_gb300 as vt

    img = _img(w, h, seed=11 * w + h)
    L = _levels_for(w, h)
    ref = oracle.build_pyramid(img, L)
    pitch = (w + 15) // 16 * 16

    def slot():
        buf = torch.zeros(pitch * h + 64, dtype=torch.uint8, device="cuda")
        v = buf[:pitch * h].view(h, pitch)[:, :w]
        v.copy_(torch.from_numpy(img))
        return v

    va, vb = slot(), slot()
    a = vt.vt_pyramid_create_on(va, L)
    b = vt.vt_pyramid_create_on(vb, L)
    assert a.level(0).data_ptr() == va.data_ptr() and a.level(0).stride(0) == pitch
    vt.vt_pyramid_build_grad(va, L, vt.VT_GRAD_S16, out=a)
    batch = vt.Batch(2, 1)
    vt.vt_batch_set(batch, [vt.frame_job(vb, b)], [], vt.KltParams(levels=L))
    vt.vt_batch_run(batch)
    torch.cuda.synchronize()
    for p in (a, b):
        for l in range(L):
            assert np.array_equal(p.level(l).cpu().numpy(), ref.levels[l]), l
            g = p.grad(l).cpu().numpy()
            assert np.array_equal(g[..., 0], ref.gx[l]) and np.array_equal(g[..., 1], ref.gy[l]), l
    if min(w, h) >= 64:  # tracking on the caller-level-0 pyramids equals tracking on owned ones
        own = vt.vt_pyramid_build_grad(img, L, vt.VT_GRAD_S16)
        rng = np.random.Generator(np.random.PCG64(w + h))
        pts = torch.from_numpy(rng.uniform([0, 0], [w - 1, h - 1], (300, 2)).astype(np.float32)).cuda()
        prm = vt.KltParams(levels=L)
        outs = []
        for p0, p1 in ((a, b), (own, own)):
            o = torch.zeros_like(pts)
            st = torch.zeros(300, dtype=torch.uint8, device="cuda")
            vt.vt_klt_track_fb(p0, p1, pts, prm, o, st)
            torch.cuda.synchronize()
            outs.append((o.cpu().numpy(), st.cpu().numpy()))
        assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][0], outs[1][0])
        own.free()
    batch.free()
    a.free()
    b.free()
    assert np.array_equal(va.cpu().numpy(), img)  # freeing the pyramid left the caller's buffer alone
    buf = torch.zeros(pitch * h + 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(vt.VTError):  # too few readable bytes after the last row
        vt.vt_pyramid_create_on(buf[:pitch * h].view(h, pitch)[:, :w], L, nbytes=pitch * h + 16)
    if pitch > 16:
        with pytest.raises(vt.VTError):  # pitch not a multiple of 16
            vt.vt_pyramid_create_on(buf[:(pitch - 8) * h].view(h, pitch - 8)[:, :min(w, pitch - 8)], L)
    with pytest.raises(vt.VTError):  # level 0 not 16-byte aligned
        vt.vt_pyramid_create_on(buf[8:8 + pitch * h].view(h, pitch)[:, :w], L)
