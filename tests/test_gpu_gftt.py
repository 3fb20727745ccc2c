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
