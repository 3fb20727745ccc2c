"""Pins of the track-bookkeeping oracle (no GPU).

The greedy thinning is pinned by the two properties that characterise it
uniquely (every kept survivor has no kept higher-priority survivor within
min_dist; every dropped one has one), checked by brute force; identity
carry-over, ageing, the cap and the identity counter by hand-built cases."""

import numpy as np

from oracle import tracks as T


def _pool(pts, ids, ages, next_id):
    return T.Pool(np.asarray(pts, np.float32).reshape(-1, 2), np.asarray(ids, np.int32), np.asarray(ages, np.int32),
                  next_id)


def test_carry_keeps_identities_ages_and_orders_by_age():
    p = _pool([[10, 10], [50, 50], [90, 90], [130, 130]], [7, 3, 9, 4], [1, 5, 5, 2], 10)
    tracked = np.array([[11, 10], [51, 49], [91, 90], [129, 131]], np.float32)
    r = T.carry(p, tracked, [1, 1, 0, 1], min_dist=5)
    assert list(r.ids) == [3, 4, 7]  # ages 6, 3, 2 after the step
    assert list(r.ages) == [6, 3, 2]
    assert np.array_equal(r.pts, tracked[[1, 3, 0]])
    assert r.next_id == 10


def test_thinning_prefers_older_then_lower_index_and_is_strict():
    p = _pool([[0, 0], [0, 0], [0, 0], [0, 0]], [1, 2, 3, 4], [1, 3, 3, 1], 5)
    # survivors 1 and 2 (same age) 4 px apart, 0 and 1 at 3 px, 3 exactly 5 px from 2
    tracked = np.array([[100, 100], [100, 103], [104, 103], [104, 108]], np.float32)
    r = T.carry(p, tracked, [1, 1, 1, 1], min_dist=5)
    # priority: index 1 (age 4), index 2 (age 4), index 0 (age 2), index 3 (age 2)
    # 1 kept; 2 at distance 4 < 5 dropped; 0 at distance 3 from 1 dropped; 3 at distance 5 from 2 (dropped)
    # and sqrt(16 + 25) from 1: kept
    assert list(r.ids) == [2, 4]


def test_spawn_fills_to_cap_in_order_with_new_identities():
    p = _pool([[5, 5]], [42], [3], 100)
    corners = np.array([[10, 10], [20, 20], [30, 30], [40, 40]], np.float32)
    r = T.spawn(p, corners, [1, 0, 1, 1], cap=3)
    assert list(r.ids) == [42, 100, 101]
    assert list(r.ages) == [3, 1, 1]
    assert np.array_equal(r.pts[1:], corners[[0, 2]])
    assert r.next_id == 102
    full = T.spawn(r, corners, None, cap=3)
    assert list(full.ids) == list(r.ids) and full.next_id == 102
    first = T.spawn(T.empty_pool(), corners, None, cap=10)  # initialisation: every detection starts a track
    assert list(first.ids) == [0, 1, 2, 3] and list(first.ages) == [1, 1, 1, 1]


def _greedy_properties(pool, tracked, status, min_dist, r):
    ok = np.nonzero(np.asarray(status) != 0)[0]
    prio = sorted(ok, key=lambda i: (-(int(pool.ages[i]) + 1), int(np.nonzero(ok == i)[0][0])))
    kept_ids = set(int(x) for x in r.ids)
    kept = [i for i in prio if int(pool.ids[i]) in kept_ids]
    md2 = np.float32(min_dist) ** 2

    def close(a, b):
        d = tracked[a].astype(np.float32) - tracked[b].astype(np.float32)
        return np.float32(d[0] * d[0]) + np.float32(d[1] * d[1]) < md2

    for n, i in enumerate(prio):
        higher_kept = [j for j in prio[:n] if j in kept]
        conflict = any(close(i, j) for j in higher_kept)
        assert (i in kept) == (not conflict)


def test_thinning_is_the_greedy_selection_brute_force():
    rng = np.random.Generator(np.random.PCG64(3))
    for trial in range(20):
        n = int(rng.integers(1, 300))
        pool = _pool(rng.uniform(0, 200, (n, 2)), rng.permutation(1000)[:n], rng.integers(1, 6, n), 1000)
        tracked = (pool.pts + rng.normal(0, 1, (n, 2))).astype(np.float32)
        status = (rng.random(n) > 0.2).astype(np.uint8)
        md = float(rng.choice([1.0, 5.0, 12.5]))
        r = T.carry(pool, tracked, status, md)
        _greedy_properties(pool, tracked, status, md, r)
        # kept survivors are min_dist apart and in priority order
        d = np.hypot(*(r.pts[:, None, :] - r.pts[None, :, :]).transpose(2, 0, 1))
        np.fill_diagonal(d, np.inf)
        assert (d >= md - 1e-4).all()
        assert (np.diff(r.ages) <= 0).all()


def test_invariants_over_a_sequence():
    rng = np.random.Generator(np.random.PCG64(9))
    pool, cap = T.empty_pool(), 120
    seen = set()
    for step in range(12):
        n = len(pool.ids)
        if n:
            tracked = (pool.pts + rng.normal(0, 2, (n, 2))).astype(np.float32)
            pool = T.carry(pool, tracked, (rng.random(n) > 0.1).astype(np.uint8), 6.0)
        corners = rng.uniform(0, 300, (200, 2)).astype(np.float32)
        before = set(int(x) for x in pool.ids)
        nid = pool.next_id
        pool = T.spawn(pool, corners, (rng.random(200) > 0.3).astype(np.uint8), cap)
        ids = [int(x) for x in pool.ids]
        assert len(ids) == len(set(ids)) <= cap
        new = set(ids) - before
        assert new == set(range(nid, pool.next_id)) and not (new & seen)
        seen |= set(ids)
        assert (pool.ages >= 1).all()


def test_thinning_threshold_is_strict():
    """Survivors exactly min_dist apart (3-4-5 triangle, exact in single
    precision) are both kept; a hair closer, only the older one."""
    p = _pool([[0, 0], [0, 0]], [1, 2], [2, 1], 3)
    r = T.carry(p, np.array([[10, 10], [13, 14]], np.float32), [1, 1], min_dist=5)
    assert list(r.ids) == [1, 2]
    r = T.carry(p, np.array([[10, 10], [13, 13.99]], np.float32), [1, 1], min_dist=5)
    assert list(r.ids) == [1]
