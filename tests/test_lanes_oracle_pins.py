"""Pins of the FP64 lane-geometry oracle (prediction with lane projection,
paper Sec. IV-B / V-C): closed forms on straight and circular lanes, brute
force against a dense sampling of the centre line, round trips, assignment
ties, the rollout state and the displacement metrics by hand."""
import math

import numpy as np

from oracle import lanes as G


def straight(n=11, length=100.0, y=0.0):
    x = np.linspace(0.0, length, n)
    return np.stack([x, np.full(n, y)], axis=1)


def test_straight_lane_closed_form():
    xy = straight()
    s, d, dist = G.project(xy, (37.5, 2.0))
    assert abs(s - 37.5) < 1e-12 and abs(d - 2.0) < 1e-12 and abs(dist - 2.0) < 1e-12
    s, d, _ = G.project(xy, (37.5, -3.0))
    assert abs(s - 37.5) < 1e-12 and abs(d + 3.0) < 1e-12
    s, d, dist = G.project(xy, (-5.0, 1.0))       # before the start: clamped to the first point
    assert s == 0.0 and abs(dist - math.sqrt(26.0)) < 1e-12 and d > 0
    s, _, _ = G.project(xy, (130.0, 0.0))          # beyond the end
    assert abs(s - 100.0) < 1e-12


def test_circular_lane():
    R, n = 50.0, 1001
    th = np.linspace(0.0, math.pi / 2, n)
    xy = np.stack([R * np.cos(th), R * np.sin(th)], axis=1)   # counter-clockwise: the centre is on the left
    rng = np.random.default_rng(0)
    for _ in range(50):
        a = rng.uniform(0.05, math.pi / 2 - 0.05)
        r = rng.uniform(40.0, 60.0)
        s, d, _ = G.project(xy, (r * math.cos(a), r * math.sin(a)))
        # inside a chord the foot point moves r sin(phi) where the arc moves
        # R phi (|phi| <= half the chord angle): |r - R| dtheta / 2 + O(dtheta^2)
        bound = abs(r - R) * (math.pi / 2 / (n - 1)) / 2 + 1e-4
        assert abs(s - R * a) < bound, (s, R * a, bound)
        assert abs(d - (R - r)) < 1e-3, (d, R - r)


def test_brute_force_dense_sampling():
    rng = np.random.default_rng(1)
    for _ in range(10):
        m = rng.integers(3, 12)
        xy = np.cumsum(rng.normal(0, 10, size=(m, 2)), axis=0)
        c = G.cumlen(xy)
        ss = np.linspace(0, c[-1], 200001)
        pts = np.array([G.unproject(xy, s) for s in ss[::100]])
        # dense samples by linear interpolation per segment (independent of unproject)
        dense = np.concatenate([np.linspace(xy[k], xy[k + 1], 2001) for k in range(m - 1)])
        for _ in range(20):
            q = xy.mean(0) + rng.normal(0, 15, size=2)
            s, d, dist = G.project(xy, q)
            dd = np.sqrt(((dense - q) ** 2).sum(1))
            assert abs(dist - dd.min()) < 0.02
            assert abs(abs(d) - dist) < 1e-12
        assert np.all(np.isfinite(pts))


def test_round_trip():
    rng = np.random.default_rng(2)
    xy = np.cumsum(rng.uniform(1.0, 5.0, size=(30, 2)), axis=0)
    xy[:, 1] += 10 * np.sin(xy[:, 0] / 20)
    c = G.cumlen(xy)
    for s in rng.uniform(0, c[-1], 200):
        p = G.unproject(xy, s)
        s2, d2, _ = G.project(xy, p)
        assert abs(s2 - s) < 1e-9 and abs(d2) < 1e-9


def test_unproject_extrapolates_linearly():
    xy = straight()
    np.testing.assert_allclose(G.unproject(xy, -5.0), [-5.0, 0.0], atol=1e-12)
    np.testing.assert_allclose(G.unproject(xy, 107.0), [107.0, 0.0], atol=1e-12)
    xy2 = np.array([[0, 0], [0, 0], [3, 4], [3, 4], [6, 8]], float)    # repeated points are skipped
    np.testing.assert_allclose(G.unproject(xy2, 7.5), [4.5, 6.0], atol=1e-12)


def test_assignment_and_ties():
    lanes = [straight(y=0.0), straight(y=4.0), straight(y=-10.0)]
    assert G.assign(lanes, (10.0, 1.0), [0, 1, 2])[0] == 0
    assert G.assign(lanes, (10.0, 3.0), [0, 1, 2])[0] == 1
    assert G.assign(lanes, (10.0, 2.0), [0, 1, 2])[0] == 0       # tie: the lowest index
    assert G.assign(lanes, (10.0, 2.0), [1, 0])[0] == 0          # index into the candidate list
    assert G.assign(lanes, (10.0, -8.0), [0, 1, 2])[0] == 2


def test_rollout_state():
    s = np.array([[0.0, 5.0], [1.0, 4.0], [2.5, 3.0]])
    p, v = G.rollout_state(s, 1, 2, 0.1)
    np.testing.assert_allclose(p, [2.5, 3.0])
    np.testing.assert_allclose(v, [15.0, 0.0])             # a backwards difference gives 0
    p, v = G.rollout_state(s, 0, 2, 0.5)
    np.testing.assert_allclose(v, [2.5, 0.0])


def test_displacement_metrics():
    true = np.zeros((4, 2, 2))
    pred = np.zeros((4, 2, 2))
    pred[:, 0, 0] = [0.0, 1.0, 2.0, 3.0]
    pred[:, 1, 1] = [1.0, 1.0, 1.0, 1.0]
    ade, fde, miss, (mA, mF, mM) = G.displacement_metrics(pred, true, 2.0)
    np.testing.assert_allclose(ade, [1.5, 1.0])
    np.testing.assert_allclose(fde, [3.0, 1.0])
    assert list(miss) == [True, False]
    assert abs(mA - 1.25) < 1e-15 and abs(mF - 2.0) < 1e-15 and mM == 0.5
