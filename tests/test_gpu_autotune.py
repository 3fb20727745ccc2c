"""The schedule tuner on the GPU: every candidate launch shape and task order
gives bit-identical tracking results, and the tuner returns a schedule."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_launch_shapes_do_not_change_results_and_tuner_picks_one():
    import torch

    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.autotune import CANDIDATES, autotune
    from paper_2607_01757_gb300.engine import BatchedTracker

    specs = [sp for sp in synth.make_stream_mix(10, seed=9) if sp.w <= 960][:4]
    frames = [synth.render_stream_frames(sp, 2) for sp in specs]
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    tr = BatchedTracker(specs, vt.KltParams())
    sids = list(range(len(specs)))
    L = [[dev(f.left[k]) for f in frames] for k in range(2)]
    R = [[dev(f.right[k]) for f in frames] for k in range(2)]
    K = [[dev(f.kps[k]) for f in frames] for k in range(2)]
    N = [[len(f.kps[k]) for f in frames] for k in range(2)]

    def one_step():  # frame 1 after frame 0, from the same pyramids every time
        tr.stage(tr.step_tables(sids, N[0], N[1], L[1], R[1], kpt=K[0], kps=K[1]))
        tr.run(graph=True)

    tr.stage(tr.step_tables(sids, [0] * len(sids), [0] * len(sids), L[0], R[0]))
    tr.run(graph=False)
    tr.advance(sids)
    ref = None
    for w, c in CANDIDATES:
        vt.vt_batch_config(tr.batch, w, c, 0)
        one_step()
        torch.cuda.synchronize()
        out = [t.cpu().numpy().tobytes() for s in tr.streams for t in (s.out_t + s.out_s)]
        if ref is None:
            ref = out
        assert out == ref, (w, c)

    def run_step():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        one_step()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # the cost-first task order gives the same results too
    tr.task_order = "cost"
    vt.vt_batch_config(tr.batch, 4, 0, 0)
    one_step()
    torch.cuda.synchronize()
    assert [t.cpu().numpy().tobytes() for s in tr.streams for t in (s.out_t + s.out_s)] == ref
    best, report = autotune(tr, run_step, reps=2, warmup=1, sms=torch.cuda.get_device_properties(0).multi_processor_count)
    assert best["shape"] in CANDIDATES and best["order"] in ("stream", "cost")
    assert set(report["knobs"]) == {"shape", "order", "pyr_ctas_per_sm"} and report["tuned_ms"] > 0
    tr.free()
