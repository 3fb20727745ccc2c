"""The tracking entry point that allocates no device memory
(vt_klt_track_tasks_noalloc), for callers that cannot allocate when they
call: real-time loops that must not wait on the allocator, and hosts that own
all device memory and forbid allocation by the code they call.  It must give
the results of the existing fused forward-backward call, twice in a row,
since every call reuses the same fixed device array, and it must leave the
device's free memory unchanged.  This file is collected last."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _setup():
    import torch

    import paper_2607_01757_gb300 as vt

    prm = vt.KltParams(win=21, levels=4, max_iters=30, eps=0.01, fb_thr=0.5)
    c = synth.make_config1(1)
    seq = synth.make_stereo_sequence(seed=2, n_frames=2, w=376, h=240, n_kp=300)
    # (I, J, points, device-side count or None): the last task takes its
    # point count from device memory and tracks only the first 111 points
    pairs = [(c.I, c.J, c.pts, None), (seq.left[0], seq.left[1], seq.kps[0], None),
             (seq.left[1], seq.right[1], seq.kps[1], None), (seq.left[0], seq.left[1], seq.kps[0], 111)]
    keep, tasks, refs = [], [], []
    for I, J, pts, n_dev in pairs:
        pI = vt.vt_pyramid_build_grad(I, 4)
        pJ = vt.vt_pyramid_build_grad(J, 4)
        n = len(pts)
        p0 = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
        out = torch.zeros((n, 2), device="cuda")
        st = torch.zeros(n, dtype=torch.uint8, device="cuda")
        err = torch.zeros(n, device="cuda")
        # the existing entry point gives the expected results
        m = n if n_dev is None else n_dev
        r_out, r_st, r_err = torch.zeros_like(out), torch.zeros_like(st), torch.zeros_like(err)
        vt.vt_klt_track_fb(pI, pJ, p0[:m], prm, r_out[:m], r_st[:m], r_err[:m])
        cnt = None
        if n_dev is not None:
            cnt = torch.tensor([n_dev], dtype=torch.int32, device="cuda")
        keep += [pI, pJ, p0, cnt]
        tasks.append(vt.track_task(pI, pJ, p0, out, st, err, fb=True, n_dev=cnt))
        refs.append((m, out, st, err, r_out, r_st, r_err))
    torch.cuda.synchronize()
    return vt, prm, keep, tasks, refs


def _check(refs, call):
    for m, out, st, err, r_out, r_st, r_err in refs:
        assert (st[m:] == 7).all(), f"call {call}: points beyond the device-side count were written"
        st, out, err = st[:m], out[:m], err[:m]
        r_st, r_out, r_err = r_st[:m], r_out[:m], r_err[:m]
        assert (st == r_st).all(), f"call {call}: status differs"
        ok = r_st.bool()
        assert (out[ok] - r_out[ok]).abs().max().item() <= 1e-5, f"call {call}: points differ"
        assert (err[ok] - r_err[ok]).abs().max().item() <= 1e-4, f"call {call}: errors differ"
        assert ok.float().mean().item() > 0.5


def test_noalloc_matches_fused_call_twice():
    import torch

    vt, prm, keep, tasks, refs = _setup()
    for call in range(2):
        for _, out, st, err, *_ in refs:
            out.fill_(-1.0)
            st.fill_(7)
            err.fill_(-1.0)
        vt.vt_klt_track_tasks_noalloc(tasks, prm)
        torch.cuda.synchronize()
        _check(refs, call)


def test_noalloc_leaves_device_memory_unchanged():
    """After a first call (which may load the kernels), further calls change
    neither torch's allocation nor the device's free memory."""
    import torch

    vt, prm, keep, tasks, refs = _setup()
    vt.vt_klt_track_tasks_noalloc(tasks, prm)
    torch.cuda.synchronize()
    a0, f0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(3):
        vt.vt_klt_track_tasks_noalloc(tasks, prm)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == a0
    assert torch.cuda.mem_get_info()[0] == f0
    for _, out, st, err, *_ in refs:
        st[:].fill_(7)
    vt.vt_klt_track_tasks_noalloc(tasks, prm)
    torch.cuda.synchronize()
    _check(refs, "after the memory check")


def test_noalloc_rejects_more_tasks_than_the_fixed_table():
    vt, prm, keep, tasks, refs = _setup()
    with pytest.raises(vt.VTError) as e:
        vt.vt_klt_track_tasks_noalloc(tasks * 65, prm)  # 260 tasks > 256
    assert e.value.code == vt.VT_ERR_ARG
