"""Track bookkeeping oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU legs)
may import this module.  It shares no code with the CUDA library.

What it computes: the identity bookkeeping of the LK front-end around the
tracker.  The paper describes it for its matching front-end (Sec. III-C:
the first frame's detections all start new tracks; later, associated
features keep their cached identities while unassociated detections start new
ones) and reports it for the LK front-end (Sec. V-A: in stereo mode only
features passing the cross-camera flow check enter the temporal pool; in mono
the pool carries itself over, about 95 % of features per frame), with the
feature cap of Sec. IV (256 keypoints).  Reading (the paper fixes no further
detail; this follows the VINS-Fusion tracker the LK front-end inherits):

* carry   the previous features whose temporal track succeeded (status 1)
          keep their identity, take their tracked position and age + 1;
* thin    survivors in order of age (descending; ties: smaller previous
          index first) are kept when no already kept survivor lies at squared
          distance < min_dist^2 (single precision, as dx*dx + dy*dy); the
          kept survivors, in that order, open the new pool;
* spawn   new detections (already in the detector's priority order, masked
          by the kept survivors) that are accepted (stereo: they passed the
          cross-camera check; mono: all) fill the pool up to `cap` in that
          order, with identities next_id, next_id + 1, ... and age 1.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Pool:
    pts: np.ndarray  # float32 [n, 2]
    ids: np.ndarray  # int32 [n]
    ages: np.ndarray  # int32 [n]
    next_id: int


def empty_pool() -> Pool:
    return Pool(np.zeros((0, 2), np.float32), np.zeros(0, np.int32), np.zeros(0, np.int32), 0)


def carry(pool: Pool, tracked, status, min_dist: float) -> Pool:
    """Survivors of a temporal step, thinned by age priority."""
    tracked = np.asarray(tracked, np.float32).reshape(-1, 2)[: len(pool.ids)]
    ok = np.asarray(status).reshape(-1)[: len(pool.ids)] != 0
    idx = np.nonzero(ok)[0]
    ages = pool.ages[idx].astype(np.int64) + 1
    order = sorted(range(len(idx)), key=lambda k: (-ages[k], k))  # age descending, then index
    md2 = np.float32(min_dist) * np.float32(min_dist)
    kept = []
    for k in order:
        p = tracked[idx[k]]
        good = True
        for j in kept:
            q = tracked[idx[j]]
            dx = np.float32(p[0] - q[0])
            dy = np.float32(p[1] - q[1])
            if np.float32(np.float32(dx * dx) + np.float32(dy * dy)) < md2:
                good = False
                break
        if good:
            kept.append(k)
    sel = idx[kept]
    return Pool(tracked[sel].copy(), pool.ids[sel].copy(), (pool.ages[sel] + 1).astype(np.int32), pool.next_id)


def spawn(pool: Pool, corners, accept, cap: int) -> Pool:
    """Append accepted detections (in order) up to `cap` features."""
    corners = np.asarray(corners, np.float32).reshape(-1, 2)
    acc = np.ones(len(corners), bool) if accept is None else np.asarray(accept).reshape(-1)[: len(corners)] != 0
    room = max(0, cap - len(pool.ids))
    new = corners[acc][:room]
    k = len(new)
    return Pool(np.vstack([pool.pts, new]).astype(np.float32),
                np.concatenate([pool.ids, pool.next_id + np.arange(k, dtype=np.int32)]).astype(np.int32),
                np.concatenate([pool.ages, np.ones(k, np.int32)]).astype(np.int32), pool.next_id + k)


def mask_of(pool: Pool, cap: int) -> np.ndarray:
    """The kept positions as a detector mask, padded with NaN to `cap` rows."""
    m = np.full((cap, 2), np.nan, np.float32)
    m[: len(pool.ids)] = pool.pts
    return m
