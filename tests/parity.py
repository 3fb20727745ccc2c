"""Comparison rules between the CUDA path and the FP64 oracle.

Flow: for points both sides track, |gpu - oracle| <= 0.01 px for 99.9 % of
them and <= 0.05 px for all.  Status: a disagreement is accepted only where
the oracle took one of its threshold decisions within 1e-4 of the threshold
(relative for the eigenvalue test, in pixels for the convergence, image-bound
and forward-backward tests)."""

from __future__ import annotations

import numpy as np

FLOW_TOL_999 = 0.01
FLOW_TOL_MAX = 0.05
MARGIN = 1e-4


def oracle_margin(res) -> np.ndarray:
    """Smallest decision margin per point of an oracle TrackResult / FBResult."""
    if hasattr(res, "min_margin"):
        return res.min_margin()
    return res.margin.min(axis=1)


def compare(gpu_pts, gpu_status, ref_pts, ref_status, ref_margin, label=""):
    gpu_pts = np.asarray(gpu_pts, np.float64).reshape(-1, 2)
    ref_pts = np.asarray(ref_pts, np.float64).reshape(-1, 2)
    gs = np.asarray(gpu_status).astype(bool)
    rs = np.asarray(ref_status).astype(bool)
    mism = np.nonzero(gs != rs)[0]
    bad = [int(i) for i in mism if not (ref_margin[i] < MARGIN)]
    assert not bad, f"{label}: status mismatch outside the margin rule at {bad[:10]} (margins {ref_margin[bad[:10]]})"
    both = gs & rs
    d = np.hypot(*(gpu_pts[both] - ref_pts[both]).T) if both.any() else np.zeros(0)
    stats = {
        "n": int(len(gs)),
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
