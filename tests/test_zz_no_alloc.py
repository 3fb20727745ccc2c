"""The tracking entry point that allocates no device memory
(vt_klt_track_tasks_noalloc), for callers that cannot allocate when they
call: code recorded into a CUDA graph, real-time loops that must not wait on
the allocator, hosts that own all device memory.  It must give the results of
the existing fused forward-backward call, twice in a row, since every call
reuses the same fixed device array.  This file is collected last."""

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
    pairs = [(c.I, c.J, c.pts), (seq.left[0], seq.left[1], seq.kps[0]), (seq.left[1], seq.right[1], seq.kps[1])]
    keep, tasks, refs = [], [], []
    for I, J, pts in pairs:
        pI = vt.vt_pyramid_build_grad(I, 4)
        pJ = vt.vt_pyramid_build_grad(J, 4)
        n = len(pts)
        p0 = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
        out = torch.zeros((n, 2), device="cuda")
        st = torch.zeros(n, dtype=torch.uint8, device="cuda")
        err = torch.zeros(n, device="cuda")
        # the existing entry point gives the expected results
        r_out, r_st, r_err = torch.zeros_like(out), torch.zeros_like(st), torch.zeros_like(err)
        vt.vt_klt_track_fb(pI, pJ, p0, prm, r_out, r_st, r_err)
        keep += [pI, pJ, p0]
        tasks.append(vt.track_task(pI, pJ, p0, out, st, err, fb=True))
        refs.append((out, st, err, r_out, r_st, r_err))
    torch.cuda.synchronize()
    return vt, prm, keep, tasks, refs


def test_noalloc_matches_fused_call_twice():
    import torch

    vt, prm, keep, tasks, refs = _setup()
    for call in range(2):
        for out, st, err, *_ in refs:
            out.fill_(-1.0)
            st.fill_(7)
            err.fill_(-1.0)
        vt.vt_klt_track_tasks_noalloc(tasks, prm)
        torch.cuda.synchronize()
        for out, st, err, r_out, r_st, r_err in refs:
            assert torch.equal(st, r_st), f"call {call}: status differs"
            ok = r_st.bool()
            assert (out[ok] - r_out[ok]).abs().max().item() <= 1e-5, f"call {call}: points differ"
            assert (err[ok] - r_err[ok]).abs().max().item() <= 1e-4, f"call {call}: errors differ"
            assert ok.float().mean().item() > 0.5


def test_noalloc_rejects_more_tasks_than_the_fixed_table():
    vt, prm, keep, tasks, refs = _setup()
    with pytest.raises(vt.VTError) as e:
        vt.vt_klt_track_tasks_noalloc(tasks * 86, prm)  # 258 tasks > 256
    assert e.value.code == vt.VT_ERR_ARG
