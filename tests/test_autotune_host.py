"""The launch-shape tuner's host logic (no GPU): it keeps the fastest shape by
median, applies it, and caches it per device and workload."""

import types

import paper_2607_01757_gb300.autotune as at


def _fake_tracker():
    s = [types.SimpleNamespace(w=752, h=480, stereo=True, levels=5),
         types.SimpleNamespace(w=640, h=480, stereo=False, levels=4)]
    return types.SimpleNamespace(streams=s, params=types.SimpleNamespace(win=21), grad_type=1, batch=object())


def test_pick_uses_the_median():
    t = {(4, 0): [1.0, 9.0, 1.1], (8, 0): [1.05, 1.05, 1.05], (4, 3): [2.0, 0.5, 2.1]}
    assert at.pick(t) == (8, 0)  # medians 1.1, 1.05, 2.0: one slow outlier does not decide
    t[(4, 0)] = [1.0, 9.0, 1.0]
    assert at.pick(t) == (4, 0)


def test_autotune_applies_and_caches(tmp_path, monkeypatch):
    applied = []
    monkeypatch.setattr(at.vt, "vt_batch_config", lambda b, w, c, p: applied.append((w, c)))
    times = {(4, 0): 2.0, (8, 0): 1.5, (4, 3): 1.7}

    def run_step():
        return times[applied[-1]]

    cache = tmp_path / "tune.json"
    tr = _fake_tracker()
    best, timings = at.autotune(tr, run_step, candidates=tuple(times), reps=3, warmup=1, cache_path=str(cache),
                                device_name="GB300")
    assert best == (8, 0) and applied[-1] == (8, 0)
    assert set(timings) == {"4x0", "8x0", "4x3"}
    applied.clear()
    best2, _ = at.autotune(tr, lambda: 1 / 0, candidates=tuple(times), cache_path=str(cache), device_name="GB300")
    assert best2 == (8, 0) and applied == [(8, 0)]  # from the cache: no step was run
    applied.clear()
    best3, _ = at.autotune(tr, run_step, candidates=tuple(times), reps=1, warmup=0, cache_path=str(cache),
                           device_name="other")
    assert best3 == (8, 0) and len(applied) == 4  # another device: tuned again
