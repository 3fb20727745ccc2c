"""Schedule tuning of the batched run.

How fast one batched step runs depends on choices that do not change any
result (every point is tracked by the same per-warp code, every pyramid
tile by the same per-CTA code):

* ``shape``: warps per CTA of the persistent tracking launch (4 or 8) and
  CTAs per SM (0 = as many as fit);
* ``order``: the order of the tasks in the tracking launch's work queue --
  as the streams are listed, or costliest first (most pyramid levels, then
  most points), so that cheap points fill the launch's tail;
* ``pyr_ctas_per_sm``: CTAs per SM of the persistent pyramid launches
  (0 = as many as fit).

The tuner times the caller's own step under each value of one knob at a
time, the others at their best so far (coordinate descent, median of a few
runs), applies the fastest schedule, re-times the default schedule and the
pick side by side, and can cache the pick per device and workload signature
in a JSON file.
"""

from __future__ import annotations

import json
import os
import statistics

from . import vt

# (warps per CTA, CTAs per SM; 0 = as many as fit)
CANDIDATES = ((4, 0), (8, 0), (4, 3), (8, 1), (4, 2))
KNOBS = {
    "shape": CANDIDATES,
    "order": ("stream", "cost"),
    "pyr_ctas_per_sm": (0, 2, 3),
}
DEFAULT = {"shape": (4, 0), "order": "stream", "pyr_ctas_per_sm": 0}


def signature(tracker) -> str:
    """Workload key: stream shapes, stereo flags, levels, window, gradient storage."""
    shapes = sorted((s.w, s.h, int(s.stereo), s.levels) for s in tracker.streams)
    return f"{len(shapes)}|{shapes}|win{tracker.params.win}|grad{tracker.grad_type}"


def pick(timings: dict):
    """The candidate with the smallest median time (ties: the first listed)."""
    best, best_t = None, float("inf")
    for cand, ts in timings.items():
        t = statistics.median(ts)
        if t < best_t:
            best, best_t = cand, t
    return best


def apply(tracker, cfg: dict, sms: int) -> None:
    """Set a schedule on the tracker (takes effect at its next staged run)."""
    w, c = cfg["shape"]
    p = cfg["pyr_ctas_per_sm"]
    vt.vt_batch_config(tracker.batch, w, c, p * sms if p else 0)
    tracker.task_order = cfg["order"]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _key(v):
    return f"{v[0]}x{v[1]}" if isinstance(v, tuple) else str(v)


def autotune(tracker, run_step, knobs=None, reps: int = 5, warmup: int = 2, cache_path=None,
             device_name: str = "", sms: int = 1):
    """Time `run_step()` (stages and runs one batched step of `tracker`,
    returns its device time in ms) under each knob value (coordinate
    descent from DEFAULT); apply and return the fastest schedule (a dict like
    DEFAULT) and a report: per-knob medians, and the default schedule and the
    pick re-timed alternately (medians and the spread of their runs)."""
    knobs = KNOBS if knobs is None else knobs
    key = f"{device_name}|{signature(tracker)}"
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        best = dict(DEFAULT)
        for k, v in cache[key]["best"].items():
            best[k] = tuple(v) if isinstance(v, list) else v
        apply(tracker, best, sms)
        return best, cache[key].get("report", {})
    cfg = dict(DEFAULT)
    report = {"knobs": {}}
    for name, values in knobs.items():
        tk = {}
        for v in values:
            apply(tracker, dict(cfg, **{name: v}), sms)
            for _ in range(warmup):
                run_step()
            tk[v] = [run_step() for _ in range(reps)]
        cfg[name] = pick(tk)
        report["knobs"][name] = {_key(v): round(statistics.median(ts), 4) for v, ts in tk.items()}
    # the default and the pick side by side, alternating
    side = {"default": [], "tuned": []}
    for _ in range(reps):
        for label, c in (("default", DEFAULT), ("tuned", cfg)):
            apply(tracker, c, sms)
            for _ in range(max(1, warmup // 2)):
                run_step()
            side[label].append(run_step())
    apply(tracker, cfg, sms)
    for label, ts in side.items():
        report[f"{label}_ms"] = round(statistics.median(ts), 4)
        report[f"{label}_spread_ms"] = round(max(ts) - min(ts), 4)
    report["best"] = {k: _key(v) if isinstance(v, tuple) else v for k, v in cfg.items()}
    if cache_path:
        cache[key] = {"best": {k: list(v) if isinstance(v, tuple) else v for k, v in cfg.items()}, "report": report}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return cfg, report
