"""Comparison rules between the CUDA path and the FP64 oracle.

Flow: for points both sides track, |gpu - oracle| <= 0.01 px for 99.9 % of
them and <= 0.05 px for all.

Status: a disagreement is excused only by the decision that produced it: the
kind of test named by the losing side's reason (the GPU's reason when the GPU
lost the point, the oracle's when the oracle did) must have been taken by
the oracle within 1e-4 of its threshold -- relative for the eigenvalue test,
in pixels for the image-bound and forward-backward tests.  An input rejection
is exact and never excused.  At most 0.1 % of the points may be excused."""

from __future__ import annotations

import numpy as np

import oracle

FLOW_TOL_999 = 0.01
FLOW_TOL_MAX = 0.05
MARGIN = 1e-4
MAX_EXCUSED_FRAC = 0.001


def _decision_margins(ref):
    return {r: ref.decision_margin(r) for r in (oracle.LOST_EIG, oracle.LOST_OOB, oracle.LOST_FB)}


def compare(gpu_pts, gpu_status, gpu_reason, ref, label="", idx=None):
    """Compare GPU results with an oracle TrackResult or FBResult (forward
    positions for FB).  ``idx`` selects the GPU entries that correspond to the
    oracle's points (a sample re-tracked by the oracle)."""
    gpu_pts = np.asarray(gpu_pts, np.float64).reshape(-1, 2)
    gpu_status = np.asarray(gpu_status)
    gpu_reason = np.asarray(gpu_reason)
    if idx is not None:
        gpu_pts, gpu_status, gpu_reason = gpu_pts[idx], gpu_status[idx], gpu_reason[idx]
    fb = hasattr(ref, "fwd")
    ref_pts = np.asarray(ref.fwd.pts if fb else ref.pts, np.float64).reshape(-1, 2)
    gs = gpu_status.astype(bool)
    rs = np.asarray(ref.status).astype(bool)
    assert len(gs) == len(rs), (label, len(gs), len(rs))
    margins = _decision_margins(ref)
    mism = np.nonzero(gs != rs)[0]
    bad = []
    for i in mism:
        why = int(gpu_reason[i]) if not gs[i] else int(ref.reason[i])
        m = margins[why][i] if why in margins else np.inf
        if not (m < MARGIN):
            bad.append((int(i), why, float(m)))
    assert not bad, f"{label}: status mismatch not excused by its own decision's margin (index, reason, margin): " \
                    f"{bad[:10]}"
    n = len(gs)
    assert len(mism) <= MAX_EXCUSED_FRAC * n, f"{label}: {len(mism)} of {n} points excused by the margin rule"
    both = gs & rs
    d = np.hypot(*(gpu_pts[both] - ref_pts[both]).T) if both.any() else np.zeros(0)
    stats = {
        "n": int(n),
        "tracked_gpu": int(gs.sum()),
        "tracked_ref": int(rs.sum()),
        "status_mismatch": int(len(mism)),
        "flow_max": float(d.max()) if d.size else 0.0,
        "flow_mean": float(d.mean()) if d.size else 0.0,
        "frac_over_001": float((d > FLOW_TOL_999).mean()) if d.size else 0.0,
    }
    assert stats["frac_over_001"] <= 0.001, f"{label}: {stats}"
    assert stats["flow_max"] <= FLOW_TOL_MAX, f"{label}: {stats}"
    return stats
