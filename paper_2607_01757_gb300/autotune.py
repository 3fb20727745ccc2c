"""Launch-shape tuning of the batched run.

The tracking launch of a vt_batch can run 4 or 8 warps per CTA and up to the
occupancy limit of CTAs per SM; which is fastest depends on the workload's
mix of point counts and pyramid sizes.  Results do not depend on the launch
shape (every point is tracked by the same per-warp code), so the tuner simply
times a few shapes on the caller's own step and keeps the fastest, with an
optional JSON cache keyed by device and workload signature.
"""

from __future__ import annotations

import json
import os
import statistics

from . import vt

# (warps per CTA, CTAs per SM; 0 = as many as fit)
CANDIDATES = ((4, 0), (8, 0), (4, 3), (8, 1), (4, 2))


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


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(tracker, run_step, candidates=CANDIDATES, reps: int = 5, warmup: int = 2, cache_path=None,
             device_name: str = ""):
    """Time `run_step()` (stages and runs one batched step of `tracker`,
    returns its device time in ms) under each launch shape; apply and return
    the fastest as (warps_per_cta, ctas_per_sm), with the timings."""
    key = f"{device_name}|{signature(tracker)}"
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        w, c = cache[key]["best"]
        vt.vt_batch_config(tracker.batch, w, c, 0)
        return (w, c), cache[key].get("timings", {})
    timings = {}
    for w, c in candidates:
        vt.vt_batch_config(tracker.batch, w, c, 0)
        for _ in range(warmup):
            run_step()
        timings[(w, c)] = [run_step() for _ in range(reps)]
    best = pick(timings)
    vt.vt_batch_config(tracker.batch, best[0], best[1], 0)
    if cache_path:
        cache[key] = {"best": list(best), "timings": {f"{w}x{c}": ts for (w, c), ts in timings.items()}}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return best, {f"{w}x{c}": ts for (w, c), ts in timings.items()}
