"""GFTT on the GPU (vt_gftt_detect) equals the oracle exactly: same corners
in the same order with the same single-precision scores."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _detect(img, prm, mask=None, level=0, levels=1):
    import torch

    import paper_2607_01757_gb300 as vt

    h, w = img.shape
    p = vt.vt_pyramid_build_grad(img, levels, vt.VT_GRAD_S16)
    g = vt.Gftt(w, h)
    out = torch.zeros((max(1, prm.max_corners), 2), device="cuda")
    sc = torch.zeros(max(1, prm.max_corners), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    m = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask, np.float32)).cuda()
    vt.vt_gftt_detect(g, p, level, prm, out, cnt, sc, mask=m)
    torch.cuda.synchronize()
    k = int(cnt.item())
    res = out[:k].cpu().numpy(), sc[:k].cpu().numpy()
    ref_pyr = oracle.build_pyramid(img, levels)
    ref = oracle.gftt(ref_pyr.gx[level], ref_pyr.gy[level], prm.max_corners, prm.quality, prm.min_dist,
                      prm.nms_radius, prm.block_radius, prm.border,
                      None if mask is None else np.asarray(mask, np.float32).astype(np.float64))
    g.free()
    p.free()
    return res, ref


CASES = [
    dict(max_corners=150, quality=0.01, min_dist=10, nms_radius=4, block_radius=1, border=10),
    dict(max_corners=1000, quality=0.01, min_dist=5, nms_radius=2, block_radius=1, border=5),
    dict(max_corners=8192, quality=0.0, min_dist=1, nms_radius=0, block_radius=0, border=0),
    dict(max_corners=300, quality=0.05, min_dist=30, nms_radius=4, block_radius=2, border=20),
    dict(max_corners=0, quality=0.01, min_dist=10, nms_radius=4, block_radius=1, border=10),
    # wide spacing: the top candidates alone cannot yield max_corners, so the selection runs again over all
    dict(max_corners=150, quality=0.001, min_dist=45, nms_radius=2, block_radius=1, border=3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_gftt_matches_oracle_752x480(case):
    import paper_2607_01757_gb300 as vt

    c = synth.make_config1(1)
    prm = vt.GfttParams(**CASES[case])
    (xy, sc), (rxy, rsc) = _detect(c.I, prm)
    assert np.array_equal(xy, rxy.astype(np.float32)), (len(xy), len(rxy))
    assert np.array_equal(sc.view(np.uint32), rsc.view(np.uint32))


def test_gftt_with_mask_and_other_shapes():
    import paper_2607_01757_gb300 as vt

    c = synth.make_config1(3)
    prm = vt.GfttParams(max_corners=500, min_dist=12)
    mask = c.pts[:100] + np.float32(0.375)
    (xy, sc), (rxy, rsc) = _detect(c.I, prm, mask=mask)
    assert np.array_equal(xy, rxy.astype(np.float32)) and np.array_equal(sc, rsc)
    for w, h, seed in [(97, 65, 1), (1920, 1200, 2), (333, 217, 3)]:
        tex = synth.BlobTexture(seed, extent=(-40, -40, w + 40, h + 40), n_blobs=max(10, int(400 * w * h / 361000)),
                                blob_radius_sigmas=4.0)
        img = synth.texture.quantize_u8(tex.eval_affine(w, h, np.array([[1.0, 0, 0], [0, 1.0, 0]])))
        (xy, sc), (rxy, rsc) = _detect(img, vt.GfttParams(max_corners=2000, min_dist=8))
        assert np.array_equal(xy, rxy.astype(np.float32)) and np.array_equal(sc, rsc), (w, h)


def test_gftt_on_a_coarser_level():
    import paper_2607_01757_gb300 as vt

    c = synth.make_config1(4)
    (xy, sc), (rxy, rsc) = _detect(c.I, vt.GfttParams(max_corners=200, min_dist=6, border=4), level=1, levels=3)
    assert len(xy) > 50 and np.array_equal(xy, rxy.astype(np.float32)) and np.array_equal(sc, rsc)


def test_gftt_dense_candidates_long_chains():
    """Every pixel of a noise image is a candidate (no suppression window),
    min_dist 2: neighbouring candidates conflict, so the parallel selection
    needs many rounds along chains of decreasing score."""
    import paper_2607_01757_gb300 as vt

    img = np.random.Generator(np.random.PCG64(5)).integers(0, 256, (150, 200), dtype=np.uint8)
    prm = vt.GfttParams(max_corners=8192, quality=0.0, min_dist=2, nms_radius=0, block_radius=1, border=0)
    (xy, sc), (rxy, rsc) = _detect(img, prm)
    assert len(rxy) > 2000
    assert np.array_equal(xy, rxy.astype(np.float32)) and np.array_equal(sc.view(np.uint32), rsc.view(np.uint32))


def test_gftt_more_kept_than_the_shared_memory_sort():
    """More than 16,384 corners survive the selection (min_dist 1), so the
    final ordering takes the global-memory path; the first 8,192 must still
    be the oracle's."""
    import paper_2607_01757_gb300 as vt

    img = np.random.Generator(np.random.PCG64(6)).integers(0, 256, (120, 200), dtype=np.uint8)
    prm = vt.GfttParams(max_corners=8192, quality=0.0, min_dist=1, nms_radius=0, block_radius=1, border=0)
    ref_pyr = oracle.build_pyramid(img, 1)
    full, _ = oracle.gftt(ref_pyr.gx[0], ref_pyr.gy[0], 10 ** 6, 0.0, 1, 0, 1, 0)
    assert len(full) > 16384
    (xy, sc), (rxy, rsc) = _detect(img, prm)
    assert len(xy) == 8192
    assert np.array_equal(xy, rxy.astype(np.float32)) and np.array_equal(sc.view(np.uint32), rsc.view(np.uint32))


def test_gftt_many_frames_in_one_call():
    """Frames of different shapes, masks and caps in one call equal the
    oracle frame by frame (and hence the single-frame call)."""
    import torch

    import paper_2607_01757_gb300 as vt

    rng = np.random.Generator(np.random.PCG64(8))
    shapes = [(480, 640), (120, 200), (600, 960), (33, 47), (480, 752)]
    imgs = [synth.make_config1(1).I[:h, :w] if h <= 480 and w <= 752 else
            rng.integers(0, 256, (h, w), dtype=np.uint8) for h, w in shapes]
    prm = vt.GfttParams(max_corners=0, quality=0.01, min_dist=7, nms_radius=3, block_radius=1, border=6)
    caps = [300, 8192, 1500, 5, 0]
    pyrs = [vt.vt_pyramid_build_grad(np.ascontiguousarray(im), 1, vt.VT_GRAD_S16) for im in imgs]
    g = vt.vt_gftt_create_pixels(sum(h * w for h, w in shapes))
    outs, jobs, masks = [], [], []
    for k, (p, cap) in enumerate(zip(pyrs, caps)):
        o = torch.zeros((max(1, cap), 2), device="cuda")
        sc = torch.zeros(max(1, cap), device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        mask = None
        if k == 0:
            mask = torch.from_numpy(rng.uniform(0, 600, (40, 2)).astype(np.float32)).cuda()
        masks.append(mask)
        outs.append((o, sc, n))
        jobs.append(vt.gftt_job(p, 0, o, n, cap, scores_out=sc, mask=mask))
    vt.vt_gftt_detect_many(g, jobs, prm)
    torch.cuda.synchronize()
    for k, (im, cap) in enumerate(zip(imgs, caps)):
        rp = oracle.build_pyramid(np.ascontiguousarray(im), 1)
        m = None if masks[k] is None else masks[k].cpu().numpy().astype(np.float64)
        rxy, rsc = oracle.gftt(rp.gx[0], rp.gy[0], cap, prm.quality, prm.min_dist, prm.nms_radius, prm.block_radius,
                               prm.border, m)
        o, sc, n = outs[k]
        cnt = int(n.item())
        assert cnt == len(rxy), (k, cnt, len(rxy))
        assert np.array_equal(o[:cnt].cpu().numpy(), rxy.astype(np.float32))
        assert np.array_equal(sc[:cnt].cpu().numpy().view(np.uint32), rsc.view(np.uint32))
    g.free()
    for p in pyrs:
        p.free()


def test_gftt_top_set_larger_than_shared_memory():
    """Many kept corners with few distinct scores (a periodic pattern): the
    top histogram bins hold more keys than the shared-memory sort, so the
    whole kept set is sorted in global memory; still the oracle's list."""
    import paper_2607_01757_gb300 as vt

    yy, xx = np.mgrid[0:160, 0:240]
    img = (((xx // 2) + (yy // 2)) % 2 * 200 + 20).astype(np.uint8)
    prm = vt.GfttParams(max_corners=8192, quality=0.0, min_dist=1, nms_radius=0, block_radius=1, border=0)
    (xy, sc), (rxy, rsc) = _detect(img, prm)
    assert len(rxy) == 8192
    assert np.array_equal(xy, rxy.astype(np.float32)) and np.array_equal(sc.view(np.uint32), rsc.view(np.uint32))
