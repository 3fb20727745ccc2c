"""Served loop: admission by HBM budget, continuous batching with two slots
in flight, every request completed, and each result the same alone and in
the mix."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _specs(n, seed):
    specs = synth.make_stream_mix(n, seed=seed, kp_range=(60, 200))
    for i, sp in enumerate(specs):  # small frames keep the test quick; shapes stay uneven
        sp.w, sp.h = [(320, 240), (376, 240), (480, 300), (256, 192)][i % 4]
    return specs


def test_served_mix_equals_alone_and_admission():
    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.server import Server, make_trace

    specs = _specs(8, 61)
    frames = [synth.render_stream_frames(sp, 3) for sp in specs]
    prm = vt.KltParams()
    # throughput mode: everything arrives at once, batches mix streams
    srv = Server(specs, frames, prm, budget_bytes=1 << 34)
    trace = make_trace(specs, 8 * 4, seed=7, frames_per_stream=3)
    st = srv.serve(trace, realtime=False)
    assert st.served == len(trace) and st.batches >= 4 and st.mean_batch > 1.0
    mixed = {i: tuple(t.clone() for t in srv.h_out[i]) for i in range(len(specs))}
    last = {}
    for r in trace:
        last[r.sid] = r
    srv.free()
    # each stream alone, same requests
    for sid in (0, 3, 5):
        solo = Server(specs, frames, prm, budget_bytes=1 << 34)
        reqs = [r for r in make_trace(specs, 8 * 4, seed=7, frames_per_stream=3) if r.sid == sid]
        solo.serve(reqs, realtime=False)
        counts = [last[sid].n_features, last[sid].n_stereo]
        assert counts[0] > 0 and (counts[1] > 0) == specs[sid].stereo
        # temporal results, then (stereo streams) the left->right results
        for k in range(len(mixed[sid]) // 2):
            n = counts[k]
            a_p, a_s = mixed[sid][2 * k:2 * k + 2]
            b_p, b_s = solo.h_out[sid][2 * k:2 * k + 2]
            assert np.array_equal(a_s[:n].numpy(), b_s[:n].numpy())
            ok = a_s[:n].numpy().astype(bool)
            assert np.array_equal(a_p[:n].numpy()[ok], b_p[:n].numpy()[ok])
        solo.free()


def test_admission_waits_for_budget():
    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.server import Server, make_trace

    specs = _specs(6, 67)
    frames = [synth.render_stream_frames(sp, 3) for sp in specs]
    srv = Server(specs, frames, vt.KltParams(), budget_bytes=0)
    one = max(srv.footprint)
    srv.budget = 2 * one  # room for two streams at a time
    trace = make_trace(specs, 6 * 3, seed=9, frames_per_stream=3, session=3)
    st = srv.serve(trace, realtime=False)
    assert st.served == len(trace)
    assert st.peak_bytes <= srv.budget
    assert st.admitted_max < len(specs) and st.admission_waits > 0
    srv.free()


def test_plain_serving_completes():
    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.server import Server, make_trace

    specs = _specs(4, 71)
    frames = [synth.render_stream_frames(sp, 3) for sp in specs]
    srv = Server(specs, frames, vt.KltParams(), budget_bytes=1 << 34)
    trace = make_trace(specs, 12, seed=11, frames_per_stream=3)
    st = srv.serve_plain(trace, realtime=False)
    assert st.served == 12 and st.features > 0
    srv.free()


def test_copy_async_round_trip():
    """vt_copy_async issues its copies in order on the stream: pinned host ->
    device, device -> device, device -> pinned host; zero-byte entries are
    skipped."""
    import torch

    import paper_2607_01757_gb300 as vt

    rng = np.random.Generator(np.random.PCG64(5))
    src = torch.from_numpy(rng.integers(0, 256, 100003, dtype=np.uint8)).pin_memory()
    d1 = torch.zeros(100003, dtype=torch.uint8, device="cuda")
    d2 = torch.zeros_like(d1)
    back = torch.zeros(100003, dtype=torch.uint8).pin_memory()
    vt.vt_copy_async([(d1.data_ptr(), src.data_ptr(), 100003), (0, 0, 0), (d2.data_ptr(), d1.data_ptr(), 100003),
                      (back.data_ptr(), d2.data_ptr(), 100003)])
    torch.cuda.synchronize()
    assert torch.equal(back, src)
    with pytest.raises(vt.VTError):
        vt.vt_copy_async([(0, src.data_ptr(), 16)])
