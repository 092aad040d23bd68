"""FP64 oracle of the lane-geometry steps of the training-free trajectory
prediction (paper Sec. IV-B, Sec. V-C): projecting 2-D agent positions onto
lane polylines (1-D arc length and signed lateral offset), lane assignment
by proximity, projecting 1-D arc lengths back onto the lane centre line, the
initial state of a rollout, and the displacement metrics.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
legs of the benchmark; shares nothing with the CUDA library.  Plain numpy in
float64, written from the definitions:
  * a lane is a polyline a_0 .. a_{M-1} with cumulative arc length
    c_0 = 0, c_{m+1} = c_m + |a_{m+1} - a_m|;
  * the projection of q is the closest point of the polyline: over every
    segment m the clamped parameter t = ((q - a_m) . (a_{m+1} - a_m)) /
    |a_{m+1} - a_m|^2 in [0, 1], the distance to a_m + t (a_{m+1} - a_m); the
    smallest distance wins (ties: the lowest segment); s = c_m + t |a_{m+1} -
    a_m|, d = the distance, signed positive to the left of the direction of
    travel (cross product);
  * lane assignment: the candidate lane with the smallest projection distance
    (ties: the lowest lane index);
  * back-projection of s: the point at arc length s on the centre line,
    continued along the first / last segment before 0 / beyond the end;
  * rollout initial state from two frames a < b of projected arc lengths:
    p = s_b, v = max((s_b - s_a) / ((b - a) dt), 0);
  * metrics per agent over F predicted frames: ADE = mean_f |pred_f - true_f|,
    FDE = |pred_F - true_F|, miss = FDE > threshold.
Degenerate segments (zero length) are skipped; a lane needs two distinct
points.
"""
import numpy as np


def cumlen(xy):
    xy = np.asarray(xy, dtype=np.float64)
    seg = np.sqrt(np.sum(np.diff(xy, axis=0) ** 2, axis=1))
    return np.concatenate([[0.0], np.cumsum(seg)])


def project(xy, q):
    """(s, d, distance) of point q on polyline xy (M x 2)."""
    xy = np.asarray(xy, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    c = cumlen(xy)
    best = (np.inf, 0.0, 0.0)
    for m in range(len(xy) - 1):
        a, b = xy[m], xy[m + 1]
        e = b - a
        L2 = e @ e
        if L2 == 0.0:
            continue
        t = min(max(((q - a) @ e) / L2, 0.0), 1.0)
        foot = a + t * e
        dist = np.sqrt((q - foot) @ (q - foot))
        if dist < best[0]:
            cross = e[0] * (q - a)[1] - e[1] * (q - a)[0]
            best = (dist, c[m] + t * np.sqrt(L2), dist if cross >= 0.0 else -dist)
    return best[1], best[2], best[0]


def assign(lanes, q, candidates):
    """Index (into candidates) of the lane nearest to q, and its (s, d)."""
    best = (np.inf, -1, 0.0, 0.0)
    for idx, l in enumerate(candidates):
        s, d, dist = project(lanes[l], q)
        if dist < best[0]:
            best = (dist, idx, s, d)
    return best[1], best[2], best[3]


def unproject(xy, s):
    """The point at arc length s of polyline xy (linear continuation beyond
    the ends)."""
    xy = np.asarray(xy, dtype=np.float64)
    c = cumlen(xy)
    keep = np.concatenate([[True], np.diff(c) > 0.0])
    xy, c = xy[keep], c[keep]
    if s <= 0.0:
        m = 0
    elif s >= c[-1]:
        m = len(c) - 2
    else:
        m = int(np.searchsorted(c, s, side="right") - 1)
    a, b = xy[m], xy[m + 1]
    return a + (s - c[m]) / (c[m + 1] - c[m]) * (b - a)


def rollout_state(s_rows, a, b, dt):
    """p = s[b], v = max((s[b] - s[a]) / ((b - a) dt), 0)."""
    s_rows = np.asarray(s_rows, dtype=np.float64)
    return s_rows[b].copy(), np.maximum((s_rows[b] - s_rows[a]) / ((b - a) * dt), 0.0)


def displacement_metrics(pred, true, miss_threshold=2.0):
    """pred, true: (F, N, 2).  Per agent ADE, FDE, miss and their means."""
    pred = np.asarray(pred, dtype=np.float64)
    true = np.asarray(true, dtype=np.float64)
    err = np.sqrt(np.sum((pred - true) ** 2, axis=2))
    ade = err.mean(axis=0)
    fde = err[-1]
    miss = fde > miss_threshold
    return ade, fde, miss, (ade.mean(), fde.mean(), miss.mean())
