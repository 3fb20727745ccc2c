"""The device-resident LK front-end loop (FrontEnd): the first frame's pool
equals the oracle's (its own detector, its own cross-camera check, its own
spawn) wherever no flow decision sits at a threshold, and every later pool
keeps the loop's invariants -- unique identities, at most `cap` features,
features at least min_dist apart, ages counting frames, new identities
handed out in order, and (stereo) new features that pass the cross-camera
check when tracked again on their own."""

import numpy as np
import pytest

import oracle
import synth
from oracle import tracks as T

pytestmark = pytest.mark.gpu


def _streams():
    specs = synth.make_stream_mix(12, seed=6)
    stereo = [sp for sp in specs if sp.stereo and sp.w <= 960][:2]
    mono = [sp for sp in specs if not sp.stereo and sp.w <= 960][:1]
    return stereo + mono


def test_first_frame_pool_matches_oracle():
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.frontend import FrontEnd

    specs = _streams()
    frames = [synth.render_stream_frames(sp, 1) for sp in specs]
    cap, md = 200, 10.0
    fe = FrontEnd(specs, vt.KltParams(), cap, md)
    fe.step([torch.from_numpy(f.left[0]).cuda() for f in frames],
            [torch.from_numpy(f.right[0]).cuda() if f.right[0] is not None else None for f in frames], graph=False)
    torch.cuda.synchronize()
    for k, (sp, f) in enumerate(zip(specs, frames)):
        pyr = oracle.build_pyramid(f.left[0], sp.levels)
        corners, _ = oracle.gftt(pyr.gx[0], pyr.gy[0], cap, fe.detect.quality, fe.detect.min_dist,
                                 fe.detect.nms_radius, fe.detect.block_radius, fe.detect.border)
        corners = corners.astype(np.float32)
        accept, near = None, np.zeros(len(corners), bool)
        if sp.stereo:
            r = oracle.track_fb(pyr, oracle.build_pyramid(f.right[0], sp.levels), corners, 21, sp.levels, 30, 0.01,
                                1e-4, 0.5)
            accept, near = r.status, r.min_margin() < 1e-4
        ref = T.spawn(T.empty_pool(), corners, accept, cap)
        pts, ids, ages = fe.pool(k)
        # identical up to the first corner whose cross-camera decision is at a threshold
        stop = int(np.argmax(near)) if near.any() else len(corners)
        m = int((accept[:stop] != 0).sum()) if accept is not None else min(stop, cap)
        m = min(m, cap)
        assert np.array_equal(pts[:m], ref.pts[:m]) and np.array_equal(ids[:m], ref.ids[:m]), sp
        assert (ages == 1).all()
        if not near.any():
            assert len(ids) == len(ref.ids)
    fe.free()


def test_loop_invariants_over_frames():
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.frontend import FrontEnd

    specs = _streams()
    F = 6
    frames = [synth.render_stream_frames(sp, F) for sp in specs]
    cap, md = 300, 8.0
    fe = FrontEnd(specs, vt.KltParams(), cap, md)
    prev = [None] * len(specs)
    next_id = [0] * len(specs)
    for t in range(F):
        fe.step([torch.from_numpy(f.left[t]).cuda() for f in frames],
                [torch.from_numpy(f.right[t]).cuda() if f.right[t] is not None else None for f in frames])
        torch.cuda.synchronize()
        for k, sp in enumerate(specs):
            pts, ids, ages = fe.pool(k)
            assert len(ids) == len(set(ids.tolist())) <= cap
            assert len(ids) > 0.5 * cap, (t, sp, len(ids))
            d = pts[:, None, :] - pts[None, :, :]
            d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]).astype(np.float32)
            np.fill_diagonal(d2, np.inf)
            assert d2.min() >= np.float32(md) * np.float32(md)
            new = ages == 1
            if prev[k] is not None:
                pid, page = prev[k]
                old = ~new
                assert np.isin(ids[old], pid).all()
                lookup = dict(zip(pid.tolist(), page.tolist()))
                assert all(a == lookup[i] + 1 for i, a in zip(ids[old].tolist(), ages[old].tolist()))
            assert sorted(ids[new].tolist()) == list(range(next_id[k], next_id[k] + int(new.sum())))
            next_id[k] += int(new.sum())
            prev[k] = (ids.copy(), ages.copy())
            if sp.stereo and new.any():  # new features pass the cross-camera check on their own
                p = torch.from_numpy(np.ascontiguousarray(pts[new])).cuda()
                o = torch.zeros_like(p)
                s = torch.zeros(p.shape[0], dtype=torch.uint8, device="cuda")
                vt.vt_klt_track_fb(fe._prev(k), fe.st[k]["pyr_r"], p, vt.KltParams(levels=sp.levels), o, s)
                torch.cuda.synchronize()
                assert s.cpu().numpy().all()
    fe.free()
