"""Track bookkeeping on the GPU (vt_tracks_carry / vt_tracks_spawn) against
the oracle, bit for bit: counts, positions, identities, ages, next identity
and the detector mask, for many pools in one call (empty, tiny, full at the
4096 cap, dense clusters, non-finite positions) and over a multi-step loop
whose inputs the test generates from the oracle's own state."""

import numpy as np
import pytest

from oracle import tracks as T

pytestmark = pytest.mark.gpu


def _to_gpu_pool(vt, ref: T.Pool, cap):
    import torch

    p = vt.TrackPool(cap)
    n = len(ref.ids)
    if n:
        p.pts[:n] = torch.from_numpy(ref.pts)
        p.ids[:n] = torch.from_numpy(ref.ids)
        p.ages[:n] = torch.from_numpy(ref.ages)
    p.count[0] = n
    p.next_id[0] = ref.next_id
    return p


def _check(p, ref: T.Pool, label):
    import torch

    torch.cuda.synchronize()
    n = int(p.count.item())
    assert n == len(ref.ids), (label, n, len(ref.ids))
    assert int(p.next_id.item()) == ref.next_id, label
    assert np.array_equal(p.pts[:n].cpu().numpy().view(np.uint32), ref.pts.view(np.uint32)), label
    assert np.array_equal(p.ids[:n].cpu().numpy(), ref.ids), label
    assert np.array_equal(p.ages[:n].cpu().numpy(), ref.ages), label


def _random_pool(rng, n, cap, spread=400.0, next_id=1000):
    pts = rng.uniform(0, spread, (n, 2)).astype(np.float32)
    return T.Pool(pts, rng.permutation(10 * cap + 10)[:n].astype(np.int32), rng.integers(1, 9, n).astype(np.int32),
                  next_id)


def test_carry_many_pools_match_oracle():
    import torch

    import paper_2607_01757_gb300 as vt

    rng = np.random.Generator(np.random.PCG64(1))
    cases = [(0, 16, 400.0), (1, 1, 400.0), (37, 64, 50.0), (1500, 2000, 640.0), (4096, 4096, 1920.0),
             (300, 300, 3.0)]  # the last: a dense cluster, long chains of conflicts
    for md in (1.0, 8.0, 10.5):
        pools, refs, jobs, masks, inputs = [], [], [], [], []
        for n, cap, spread in cases:
            ref = _random_pool(rng, n, cap, spread)
            tracked = (ref.pts + rng.normal(0, 0.7, (n, 2))).astype(np.float32)
            status = (rng.random(n) > 0.15).astype(np.uint8)
            if n > 40:  # non-finite survivors must neither hang nor conflict
                tracked[5] = [np.nan, 3.0]
                tracked[9] = [np.inf, -np.inf]
                status[[5, 9]] = 1
            p = _to_gpu_pool(vt, ref, cap)
            tk = torch.from_numpy(np.ascontiguousarray(tracked)).cuda() if n else torch.zeros((1, 2), device="cuda")
            st = torch.from_numpy(status).cuda() if n else torch.zeros(1, dtype=torch.uint8, device="cuda")
            mask = torch.full((cap, 2), 7.0, device="cuda")
            jobs.append(vt.carry_job(p, tk, st, mask))
            pools.append(p)
            masks.append(mask)
            inputs.append((tk, st))
            refs.append(T.carry(ref, tracked, status, md))
        vt.vt_tracks_carry(jobs, md)
        for (n, cap, _), p, ref, mask in zip(cases, pools, refs, masks):
            _check(p, ref, f"carry n={n} md={md}")
            m, rm = mask.cpu().numpy(), T.mask_of(ref, cap)
            k = len(ref.ids)
            assert np.array_equal(m[:k].view(np.uint32), rm[:k].view(np.uint32))
            assert np.isnan(m[k:]).all()


def test_spawn_many_pools_match_oracle():
    import torch

    import paper_2607_01757_gb300 as vt

    rng = np.random.Generator(np.random.PCG64(2))
    cases = [(0, 150, 200), (10, 150, 0), (149, 150, 30), (150, 150, 50), (100, 4096, 3000), (2000, 4096, 5000)]
    jobs, pools, refs = [], [], []
    for n, cap, nc in cases:
        ref = _random_pool(rng, n, cap, next_id=int(rng.integers(0, 10 ** 6)))
        corners = rng.uniform(0, 600, (max(nc, 1), 2)).astype(np.float32)
        accept = (rng.random(max(nc, 1)) > 0.25).astype(np.uint8)
        p = _to_gpu_pool(vt, ref, cap)
        c = torch.from_numpy(corners).cuda()
        cnt = torch.tensor([nc], dtype=torch.int32, device="cuda")
        a = torch.from_numpy(accept).cuda()
        jobs.append(vt.spawn_job(p, c, cnt, a))
        pools.append((p, c, cnt, a))
        refs.append(T.spawn(ref, corners[:nc], accept[:nc], cap))
    vt.vt_tracks_spawn(jobs)
    for (n, cap, nc), (p, *_), ref in zip(cases, pools, refs):
        _check(p, ref, f"spawn n={n} cap={cap} nc={nc}")
    # without an accept array every detection may spawn
    ref = _random_pool(rng, 20, 100)
    p = _to_gpu_pool(vt, ref, 100)
    corners = rng.uniform(0, 600, (300, 2)).astype(np.float32)
    c = torch.from_numpy(corners).cuda()
    cnt = torch.tensor([300], dtype=torch.int32, device="cuda")
    vt.vt_tracks_spawn([vt.spawn_job(p, c, cnt)])
    _check(p, T.spawn(ref, corners, None, 100), "spawn, all accepted")


def test_bookkeeping_loop_matches_oracle():
    """Eight steps of carry + spawn on three streams; each step's tracked
    positions, statuses and detections are drawn by the test from the
    oracle's pools, and the same arrays go to both sides."""
    import torch

    import paper_2607_01757_gb300 as vt

    rng = np.random.Generator(np.random.PCG64(3))
    caps = [150, 256, 1000]
    refs = [T.empty_pool() for _ in caps]
    pools = [vt.TrackPool(c) for c in caps]
    keep = []
    for step in range(8):
        cjobs, sjobs = [], []
        for k, cap in enumerate(caps):
            n = len(refs[k].ids)
            tracked = (refs[k].pts + rng.normal(0, 3.0, (n, 2))).astype(np.float32)
            status = (rng.random(n) > 0.08).astype(np.uint8)
            tk = torch.zeros((cap, 2), device="cuda")
            st = torch.zeros(cap, dtype=torch.uint8, device="cuda")
            if n:
                tk[:n] = torch.from_numpy(tracked)
                st[:n] = torch.from_numpy(status)
            mask = torch.zeros((cap, 2), device="cuda")
            cjobs.append(vt.carry_job(pools[k], tk, st, mask))
            refs[k] = T.carry(refs[k], tracked, status, 9.0) if n else refs[k]
            nc = int(rng.integers(0, 2 * cap))
            corners = rng.uniform(0, 752, (max(nc, 1), 2)).astype(np.float32)
            accept = (rng.random(max(nc, 1)) > 0.2).astype(np.uint8)
            c = torch.from_numpy(corners).cuda()
            cnt = torch.tensor([nc], dtype=torch.int32, device="cuda")
            a = torch.from_numpy(accept).cuda()
            sjobs.append(vt.spawn_job(pools[k], c, cnt, a))
            refs[k] = T.spawn(refs[k], corners[:nc], accept[:nc], cap)
            keep += [tk, st, mask, c, cnt, a]
        vt.vt_tracks_carry(cjobs, 9.0)
        vt.vt_tracks_spawn(sjobs)
        for k, cap in enumerate(caps):
            _check(pools[k], refs[k], f"step {step} stream {k}")


def test_track_task_device_count():
    """A tracking task with a device-side count tracks exactly its first
    *n_dev points (bit-identical to a task of that size) and leaves the rest
    of its outputs untouched."""
    import torch

    import paper_2607_01757_gb300 as vt
    import synth

    c = synth.make_config1(1)
    prm = vt.KltParams(win=21, levels=4)
    pI = vt.vt_pyramid_build_grad(c.I, 4, vt.VT_GRAD_S16)
    pJ = vt.vt_pyramid_build_grad(c.J, 4, vt.VT_GRAD_S16)
    pts = torch.from_numpy(np.ascontiguousarray(c.pts, np.float32)).cuda()
    n, k = pts.shape[0], 97
    outs = []
    for n_dev in (torch.tensor([k], dtype=torch.int32, device="cuda"), None):
        o = torch.full((n, 2), -5.0, device="cuda")
        st = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        b = vt.Batch(2, 1)
        src = pts if n_dev is not None else pts[:k]
        vt.vt_batch_set(b, [], [vt.track_task(pI, pJ, src, o, st, fb=True, n_dev=n_dev)], prm)
        vt.vt_batch_run(b)
        torch.cuda.synchronize()
        outs.append((o.cpu().numpy(), st.cpu().numpy()))
        b.free()
    (o1, s1), (o2, s2) = outs
    assert np.array_equal(o1[:k].view(np.uint32), o2[:k].view(np.uint32)) and np.array_equal(s1[:k], s2[:k])
    assert (o1[k:] == -5.0).all() and (s1[k:] == 7).all()
    pI.free()
    pJ.free()
