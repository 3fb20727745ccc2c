"""The benchmark's JSON contract.

CPU: the reference arm (the oracle timed on the host) prints one JSON line
with the contract's keys.  GPU: a small native run prints one JSON line with
every key the contract asks for, each section filled in."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "cpu_baseline", "clocks")


def _run(args, timeout):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=timeout, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--streams", "2"], 600)
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.gpu
def test_native_small_run_line():
    d = _run(["--small", "--steps", "3", "--warmup", "3", "--no-served", "--cpu-seconds", "2"], 900)
    for k in KEYS:
        assert k in d, k
    assert d["value"] > 0 and d["gpu_launches"] > 0 and d["n_gpus"] == 1
    r = d["roofline"]
    assert 0 < r["frac"] < 1.5 and r["achieved"] > 0 and r["peak"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["value"] > 0
    for sec in ("gftt", "stereo_gate", "track_bookkeeping", "frontend_loop", "plain"):
        assert d[sec], sec
    assert d["config"]["launch_shape"]["warps_per_cta"] in (4, 8)
    assert 0 < d["config"]["hbm_used_gb"] < 280


@pytest.mark.gpu
def test_precision_row():
    """The bench's precision row: int16 and FP16 gradient storage against the
    FP64 oracle on both precision workloads."""
    import torch

    import bench
    import paper_2607_01757_gb300 as vt

    d = bench.precision_against_oracle(bench.precision_gpu_runs(vt, torch))
    rows = d["rows"]
    assert set(rows) == {"blur_exposure", "high_contrast"}
    for row in rows.values():
        assert row["int16"]["max_px"] <= 0.05 and row["fp16"]["status_equal"] >= 0.99
    assert rows["high_contrast"]["fp16_rounded_window_samples"] > 1e-3
    assert rows["blur_exposure"]["fp16_rounded_window_samples"] == 0.0


def test_cpu_baseline_uses_stream_levels_and_counts_iterations():
    """The native arm's CPU baseline: the oracle on a bounded sample, each
    stream with its own level count, and the mean Newton iterations per
    level of that sample."""
    from types import SimpleNamespace

    import bench

    specs, frames = bench.make_workload(1, 2, 4, 1)
    prm = SimpleNamespace(win=21, levels=4, max_iters=30, eps=0.01, min_eig=1e-4, fb_thr=0.5)
    r = bench.cpu_baseline(specs, frames, prm, 0.5)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] == 1
    il = r["iters_per_level"]
    assert sorted(il) == [f"L{lv}" for lv in range(specs[0].levels)]
    assert all(v > 0 for v in il.values())


@pytest.mark.gpu
def test_served_sweep_rows():
    """The bench's served section on a small mix: each rate runs both arms on
    several traces; the row's p99 is the median of the runs' p99s."""
    import statistics
    from types import SimpleNamespace

    import bench
    import paper_2607_01757_gb300 as vt

    wl = bench.make_workload(6, 3, 11, 1)
    a = SimpleNamespace(served_requests=120, served_sweep_requests=60, served_reps=3, served_rates=[1.0, 4.0],
                        served_budget_gb=20.0, served_slots=2, seed=11, frames=3)
    same = lambda x: x  # noqa: E731 - one rank
    out = bench.run_served(a, wl, vt.KltParams(), lambda: None, same, same)
    assert [r["rate_x"] for r in out["sweep"]] == [1.0, 4.0]
    for row in out["sweep"]:
        for arm in ("batched", "plain"):
            r = row[arm]
            assert len(r["p99_ms_runs"]) == 3 and r["requests"] == 180
            assert abs(r["p99_ms"] - statistics.median(r["p99_ms_runs"])) < 1e-3
            assert r["features_per_s"] > 0 and r["p50_ms"] <= r["p99_ms"] + 1e-9
    assert out["batched_saturated"]["requests"] == 120 and out["plain_saturated"]["requests"] == 120
    assert set(out["best_at_p99_le_2ms"]) == {"batched", "plain"}
