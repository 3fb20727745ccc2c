"""Stereo triangulation gate on the GPU against the FP64 oracle.

Inputs: a general rig (rotation, translation with a small vertical and
forward part, different intrinsics per camera) and a mix of correspondences
that exercises every decision -- exact and noisy pairs, pairs off the
epipolar line, far points (negligible disparity), points behind a camera,
out-of-range depths, untracked and non-finite pairs -- 5,000 of them (several
blocks and a ragged tail); then the left->right pairs the oracle tracks on
the 752x480 stereo sequence.  Decisions must agree except where the oracle's
deciding value lies within 1e-6 of its threshold (both sides compute in
FP64, by different routes: SVD of A against Jacobi on A^T A); points agree to
the float32 rounding of the output.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import stereo as S

pytestmark = pytest.mark.gpu

MARGIN = 1e-6


def _rot(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    return (np.array([[cc, -sc, 0], [sc, cc, 0], [0, 0, 1]]) @ np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
            @ np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]]))


def _gpu_gate(pl, pr, st_in, rig, prm, inplace=False):
    import torch

    import paper_2607_01757_gb300 as vt

    n = len(pl)
    tl = torch.from_numpy(np.ascontiguousarray(pl, np.float32)).cuda()
    tr = torch.from_numpy(np.ascontiguousarray(pr, np.float32)).cuda()
    ts = None if st_in is None else torch.from_numpy(np.ascontiguousarray(st_in, np.uint8)).cuda()
    xyz = torch.full((n, 3), 7.0, device="cuda")
    st = ts if inplace else torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    rs = torch.full((n,), 99, dtype=torch.uint8, device="cuda")
    vt.vt_stereo_gate(tl, tr, vt.StereoRig(rig.kl, rig.kr, rig.R, rig.t),
                      vt.GateParams(prm.min_disp, prm.z_min, prm.z_max, prm.max_reproj), st, status_in=ts,
                      xyz_out=xyz, reason_out=rs)
    torch.cuda.synchronize()
    return xyz.cpu().numpy(), st.cpu().numpy(), rs.cpu().numpy()


def _compare(g, r, label):
    xyz, st, rs = g
    assert set(np.unique(st)) <= {0, 1}
    mism = np.nonzero(rs != r.reason)[0]
    bad = [int(i) for i in mism if not (r.margin[i] < MARGIN)]
    assert not bad, f"{label}: reasons differ at {bad[:8]}: gpu {rs[bad[:8]]} oracle {r.reason[bad[:8]]}"
    assert (st == (rs == S.GATE_OK)).all()
    same = rs == r.reason
    np.testing.assert_allclose(xyz[same], r.xyz[same].astype(np.float32), rtol=1e-5, atol=1e-6, err_msg=label)
    return {k: int((r.reason == v).sum()) for k, v in
            [("ok", S.GATE_OK), ("input", S.GATE_INPUT), ("disp", S.GATE_DISP), ("depth", S.GATE_DEPTH),
             ("reproj", S.GATE_REPROJ)]} | {"mismatch": int(len(mism))}


def _mixed_pairs(n=5000, seed=11):
    rng = np.random.Generator(np.random.PCG64(seed))
    rig = S.Rig(kl=(458.654, 457.296, 367.215, 248.375), kr=(457.587, 456.134, 379.999, 255.238),
                R=_rot(*rng.uniform(-0.03, 0.03, 3)), t=np.array([-0.110, 0.0004, -0.0009]))
    z = np.exp(rng.uniform(np.log(0.05), np.log(400.0), n))  # 5 cm .. 400 m: both depth limits and far points
    XL = np.stack([rng.uniform(-0.6, 0.6, n) * z, rng.uniform(-0.45, 0.45, n) * z, z], 1)
    XR = XL @ rig.R.T + rig.t
    pl = np.stack([rig.kl[0] * XL[:, 0] / XL[:, 2] + rig.kl[2], rig.kl[1] * XL[:, 1] / XL[:, 2] + rig.kl[3]], 1)
    pr = np.stack([rig.kr[0] * XR[:, 0] / XR[:, 2] + rig.kr[2], rig.kr[1] * XR[:, 1] / XR[:, 2] + rig.kr[3]], 1)
    kind = rng.integers(0, 6, n)
    noise = rng.normal(0, 0.4, (n, 2))
    pr = np.where((kind == 1)[:, None], pr + noise, pr)  # small noise
    pr = np.where((kind == 2)[:, None], pr + rng.normal(0, 3.0, (n, 2)), pr)  # off the epipolar line
    pr = np.where((kind == 3)[:, None], pr + np.array([25.0, 0.0]), pr)  # wrong match: behind / too near
    st = (rng.random(n) > 0.05).astype(np.uint8)
    pl[rng.integers(0, n, 10), 0] = np.nan
    pr[rng.integers(0, n, 10), 1] = np.inf
    return rig, pl.astype(np.float32), pr.astype(np.float32), st


def test_gate_matches_oracle_on_mixed_pairs():
    rig, pl, pr, st = _mixed_pairs()
    prm = S.GateParams(min_disp=1.0, z_min=0.1, z_max=50.0, max_reproj=1.5)
    r = S.stereo_gate(pl, pr, st, rig, prm)
    counts = _compare(_gpu_gate(pl, pr, st, rig, prm), r, "mixed")
    print("gate decisions:", counts)
    for k in ("ok", "input", "disp", "depth", "reproj"):
        assert counts[k] >= 20, counts  # every decision is exercised


def test_gate_in_place_status_and_other_parameters():
    rig, pl, pr, st = _mixed_pairs(777, seed=12)
    prm = S.GateParams(min_disp=0.0, z_min=0.5, z_max=np.inf, max_reproj=0.75)
    r = S.stereo_gate(pl, pr, st, rig, prm)
    _compare(_gpu_gate(pl, pr, st, rig, prm, inplace=True), r, "in place")
    r = S.stereo_gate(pl, pr, None, rig, prm)
    _compare(_gpu_gate(pl, pr, None, rig, prm), r, "no status")


def test_gate_on_tracked_stereo_sequence_752x480():
    """Left->right pairs tracked (with forward-backward check) by the oracle
    on the stereo sequence: rectified rig, f = 460 px, baseline 0.11 m."""
    seq = synth.make_stereo_sequence(seed=2, n_frames=1, w=752, h=480, n_kp=1000)
    pL, pR = oracle.build_pyramid(seq.left[0], 5), oracle.build_pyramid(seq.right[0], 5)
    kp = seq.kps[0]
    fb = oracle.track_fb(pL, pR, kp, 21, 5, 30, 0.01, 1e-4, 0.5)
    c = ((752 - 1) / 2.0, (480 - 1) / 2.0)
    rig = S.Rig(kl=(seq.f, seq.f, *c), kr=(seq.f, seq.f, *c), R=np.eye(3), t=np.array([-seq.baseline, 0.0, 0.0]))
    prm = S.GateParams()
    pr = fb.fwd.pts.astype(np.float32)
    r = S.stereo_gate(kp, pr, fb.status, rig, prm)
    counts = _compare(_gpu_gate(kp, pr, fb.status, rig, prm), r, "sequence")
    print("sequence gate:", counts)
    assert counts["ok"] > 0.8 * int(fb.status.sum()), counts
    # the wall sits 3-4 m away (plus bumps): kept depths say so
    z = r.xyz[r.status == 1, 2]
    assert 2.0 < np.median(z) < 6.0


def test_batched_gate_matches_single_calls_and_oracle():
    """The gate as one more launch of a batched run (stereo streams of the
    stream mix, one mono stream in the batch too): bit-identical to
    vt_stereo_gate on the same pairs, and, on a sample of points the oracle
    tracks and gates itself, the same decisions wherever neither the
    oracle's flow nor its gate decision sits near a threshold."""
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.engine import BatchedTracker

    specs = synth.make_stream_mix(12, seed=5)
    stereo = [sp for sp in specs if sp.stereo and sp.w <= 960][:3]
    mono = [sp for sp in specs if not sp.stereo][:1]
    pick = stereo + mono
    assert len(stereo) >= 2
    frames = [synth.render_stream_frames(sp, 2) for sp in pick]
    rigs = [vt.StereoRig(*synth.stream_rig(sp)) if sp.stereo else None for sp in pick]
    gprm = vt.GateParams(min_disp=1.0, z_min=0.1, z_max=50.0, max_reproj=1.5)
    prm = vt.KltParams()
    tr = BatchedTracker(pick, prm, gate=gprm, rigs=rigs)
    sids = list(range(len(pick)))
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    L0, L1 = [dev(f.left[0]) for f in frames], [dev(f.left[1]) for f in frames]
    R0, R1 = [dev(f.right[0]) for f in frames], [dev(f.right[1]) for f in frames]
    k0, k1 = [dev(f.kps[0]) for f in frames], [dev(f.kps[1]) for f in frames]
    n0, n1 = [len(f.kps[0]) for f in frames], [len(f.kps[1]) for f in frames]
    tr.stage(tr.step_tables(sids, [0] * len(sids), [0] * len(sids), L0, R0))
    tr.run(graph=False)
    tr.advance(sids)
    tr.stage(tr.step_tables(sids, n0, n1, L1, R1, kpt=k0, kps=k1))
    launches = vt.vt_batch_info(tr.batch)["launches_per_run"]
    tr.run(graph=True)
    tr.advance(sids)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(23))
    for i, sp in enumerate(stereo):
        s, f, n = tr.streams[i], frames[i], n1[i]
        st = torch.zeros(n, dtype=torch.uint8, device="cuda")
        xyz = torch.zeros((n, 3), device="cuda")
        rs = torch.zeros(n, dtype=torch.uint8, device="cuda")
        vt.vt_stereo_gate(k1[i], s.out_s[0], rigs[i], gprm, st, status_in=s.out_s[1], xyz_out=xyz, reason_out=rs)
        torch.cuda.synchronize()
        assert torch.equal(st, s.gate_out[0][:n]) and torch.equal(rs, s.gate_out[2][:n])
        assert torch.equal(xyz, s.gate_out[1][:n])
        g_st = st.cpu().numpy()
        assert g_st.sum() > 0.8 * s.out_s[1][:n].sum().item()
        # oracle: its own tracking and gate on a sample
        idx = np.sort(rng.choice(n, size=min(48, n), replace=False))
        fb = oracle.track_fb(oracle.build_pyramid(f.left[1], sp.levels), oracle.build_pyramid(f.right[1], sp.levels),
                             f.kps[1][idx], 21, sp.levels, 30, 0.01, 1e-4, 0.5)
        kl, kr, R, t = synth.stream_rig(sp)
        r = S.stereo_gate(f.kps[1][idx], fb.fwd.pts, fb.status, S.Rig(kl, kr, np.reshape(R, (3, 3)), np.array(t)),
                          S.GateParams(gprm.min_disp, gprm.z_min, gprm.z_max, gprm.max_reproj))
        near = (r.margin < 0.05) | (fb.min_margin() < 1e-4)
        bad = np.nonzero((g_st[idx] != r.status) & ~near)[0]
        assert not len(bad), (sp, bad, g_st[idx][bad], r.reason[bad])
    tr.free()
    # pyramid levels + tail + tracking + gate
    assert launches >= 4


def test_batched_gate_general_rigs_without_tracking():
    """Gate tasks alone in a batched run (no frames, no tracking tasks), each
    with its own general rig: equal to the oracle under the margin rule and
    bit-identical to the single call."""
    import torch

    import paper_2607_01757_gb300 as vt

    gprm = vt.GateParams(min_disp=0.5, z_min=0.2, z_max=80.0, max_reproj=1.5)
    prm_o = S.GateParams(0.5, 0.2, 80.0, 1.5)
    b = vt.Batch(1, 4)
    vt.vt_batch_set(b, [], [], vt.KltParams())
    tasks, keep, refs = [], [], []
    for seed in (21, 22, 23):
        rig, pl, pr, st = _mixed_pairs(600 + 37 * seed, seed=seed)
        dl, dr = torch.from_numpy(pl).cuda(), torch.from_numpy(pr).cuda()
        ds = torch.from_numpy(st).cuda()
        out = torch.zeros(len(pl), dtype=torch.uint8, device="cuda")
        xyz = torch.zeros((len(pl), 3), device="cuda")
        rs = torch.zeros(len(pl), dtype=torch.uint8, device="cuda")
        vrig = vt.StereoRig(rig.kl, rig.kr, rig.R, rig.t)
        tasks.append(vt.gate_task(dl, dr, vrig, out, status_in=ds, xyz=xyz, reason=rs))
        keep.append((dl, dr, ds, out, xyz, rs, vrig, pl, pr, st, rig))
    vt.vt_batch_set_gates(b, tasks, gprm)
    vt.vt_batch_run(b)
    torch.cuda.synchronize()
    for dl, dr, ds, out, xyz, rs, vrig, pl, pr, st, rig in keep:
        r = S.stereo_gate(pl, pr, st, rig, prm_o)
        _compare((xyz.cpu().numpy(), out.cpu().numpy(), rs.cpu().numpy()), r, "batched general rig")
        g = _gpu_gate(pl, pr, st, rig, prm_o)
        assert np.array_equal(g[1], out.cpu().numpy()) and np.array_equal(g[2], rs.cpu().numpy())
        assert np.array_equal(g[0].view(np.uint32), xyz.cpu().numpy().view(np.uint32))
    b.free()
