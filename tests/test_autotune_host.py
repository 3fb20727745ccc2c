"""The schedule tuner's host logic (no GPU): it keeps the fastest value of
each knob by median (coordinate descent), applies the pick, re-times the
default against it, and caches the pick per device and workload."""

import types

import paper_2607_01757_gb300.autotune as at


def _fake_tracker():
    s = [types.SimpleNamespace(w=752, h=480, stereo=True, levels=5),
         types.SimpleNamespace(w=640, h=480, stereo=False, levels=4)]
    return types.SimpleNamespace(streams=s, params=types.SimpleNamespace(win=21), grad_type=1, batch=object(),
                                 task_order="stream")


def test_pick_uses_the_median():
    t = {(4, 0): [1.0, 9.0, 1.1], (8, 0): [1.05, 1.05, 1.05], (4, 3): [2.0, 0.5, 2.1]}
    assert at.pick(t) == (8, 0)  # medians 1.1, 1.05, 2.0: one slow outlier does not decide
    t[(4, 0)] = [1.0, 9.0, 1.0]
    assert at.pick(t) == (4, 0)


def test_autotune_coordinate_descent_applies_and_caches(tmp_path, monkeypatch):
    applied = []
    monkeypatch.setattr(at.vt, "vt_batch_config", lambda b, w, c, p: applied.append((w, c, p)))
    tr = _fake_tracker()
    # step time: a shape term, an order term and a pyramid-grid term
    shape_t = {(4, 0): 2.0, (8, 0): 1.5, (4, 3): 1.7}
    order_t = {"stream": 0.3, "cost": 0.0}
    pyr_t = {0: 0.2, 152 * 2: 0.0, 152 * 3: 0.1}

    def run_step():
        w, c, p = applied[-1]
        return shape_t[(w, c)] + order_t[tr.task_order] + pyr_t[p]

    knobs = {"shape": tuple(shape_t), "order": ("stream", "cost"), "pyr_ctas_per_sm": (0, 2, 3)}
    cache = tmp_path / "tune.json"
    best, rep = at.autotune(tr, run_step, knobs=knobs, reps=3, warmup=1, cache_path=str(cache),
                            device_name="GB300", sms=152)
    assert best == {"shape": (8, 0), "order": "cost", "pyr_ctas_per_sm": 2}
    assert applied[-1] == (8, 0, 304) and tr.task_order == "cost"
    assert rep["default_ms"] == 2.5 and rep["tuned_ms"] == 1.5
    assert set(rep["knobs"]) == {"shape", "order", "pyr_ctas_per_sm"}
    assert rep["knobs"]["shape"]["8x0"] == 2.0  # timed with the defaults of the later knobs
    applied.clear()
    best2, _ = at.autotune(tr, lambda: 1 / 0, knobs=knobs, cache_path=str(cache), device_name="GB300", sms=152)
    assert best2 == best and applied == [(8, 0, 304)]  # from the cache: no step was run
    applied.clear()
    best3, _ = at.autotune(tr, run_step, knobs=knobs, reps=1, warmup=0, cache_path=str(cache),
                           device_name="other", sms=152)
    assert best3 == best and len(applied) > 8  # another device: tuned again
