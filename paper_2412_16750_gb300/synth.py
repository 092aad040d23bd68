"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays them out; it holds none of the
simulator's arithmetic, so both the CUDA path and the FP64 oracle can use it.
Every floating-point value it returns is exactly representable in float32
(rounded once, then widened), so the two sides start from identical inputs.

Recipe (all draws from numpy PCG64):
  * lanes are filled head first: the head of every lane sits at p = 0, each
    follower is placed behind its leader with a bumper-to-bumper gap drawn
    from U[20, 40] m; every vehicle is 5 m long;
  * initial speeds U[10, 30] m/s;
  * true parameters v0 U[25, 35], T U[1, 2], s0 U[1.5, 3], a_max U[0.8, 2],
    b U[1, 3], delta = 4;
  * observation noise N(0, 0.5^2) m, drawn here and added by the caller to a
    trajectory it computes itself.
The paper's own datasets (NGSIM US-101, a non-public Singapore set, Waymo
Open Motion) are not available; these inputs stand in for them.
"""
import numpy as np

SEED_BASE = 20241216

PARAM_NAMES = ("v0", "T", "s0", "a_max", "b", "delta")

# Ranges of the true parameters (v0, T, s0, a_max, b); delta fixed at 4.
TRUE_RANGES = ((25.0, 35.0), (1.0, 2.0), (1.5, 3.0), (0.8, 2.0), (1.0, 3.0))
DELTA = 4.0

# Zero-knowledge initial guess of Sec. IV-A: a_max 10, a_pref (b) 2, T_pref 1,
# s_min (s0) 5, v_targ (v0) 50.  Order (v0, T, s0, a_max, b, delta).
PLAIN_INIT = (50.0, 1.0, 5.0, 10.0, 2.0, 4.0)

# Boxes of Sec. IV-A in (v0, T, s0, a_max, b) order.  The a_max box is widened
# from [5, 10] to [0.5, 10] so that it contains the true range U[0.8, 2].
BOX_LO = (20.0, 0.1, 1.0, 0.5, 0.1)
BOX_HI = (60.0, 5.0, 10.0, 10.0, 5.0)

A_MIN = -10.0
LENGTH = 5.0
GAP_RANGE = (20.0, 40.0)
SPEED_RANGE = (10.0, 30.0)
NOISE_STD = 0.5


def f32(a):
    """Round to float32 and widen back to float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rng_for(config_index, salt=0):
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_index + 1000 * salt))


def lane_offsets(counts):
    counts = np.asarray(counts, dtype=np.int64)
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off.astype(np.int32)


def make_scene(counts, rng):
    """Lanes with the given vehicle counts, head first within each lane.

    Returns a dict with lane_off (int32 [L+1]), length, p_init, v_init
    (float64 [N], float32-exact) and theta_true (float64 (6, N)).
    """
    counts = np.asarray(counts, dtype=np.int64)
    lane_off = lane_offsets(counts)
    N = int(lane_off[-1])
    length = np.full(N, LENGTH)
    gaps = rng.uniform(*GAP_RANGE, size=N)
    v_init = rng.uniform(*SPEED_RANGE, size=N)
    # positions: cumulative placement behind the head of each lane
    p = np.empty(N)
    for_heads = np.zeros(N, dtype=bool)
    for_heads[lane_off[:-1][counts > 0]] = True
    step = np.where(for_heads, 0.0, gaps + LENGTH)
    csum = np.cumsum(step)
    lane_start_sum = np.repeat(csum[lane_off[:-1][counts > 0]], counts[counts > 0])
    p[:] = -(csum - lane_start_sum)
    theta = np.empty((6, N))
    for q, (lo, hi) in enumerate(TRUE_RANGES):
        theta[q] = rng.uniform(lo, hi, size=N)
    theta[5] = DELTA
    return dict(lane_off=lane_off, length=f32(length), p_init=f32(p), v_init=f32(v_init),
                theta_true=f32(theta))


def plain_init(N):
    th = np.empty((6, N))
    for q, x in enumerate(PLAIN_INIT):
        th[q] = x
    return th


def noise(rng, n_obs, N):
    return rng.normal(0.0, NOISE_STD, size=(n_obs, N))


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def config0():
    """Plain fit, small: 10 lanes x 100 vehicles, 100 steps, dt 0.1 s, all
    steps observed."""
    rng = rng_for(0)
    sc = make_scene([100] * 10, rng)
    sc.update(K=100, dt=0.1, obs_stride=1, noise=noise(rng, 100, 1000), name="10x100 K=100")
    return sc


def config1(n_lanes=20000, per_lane=100, K=1000):
    """Paper scale: 20,000 lanes x 100 vehicles (2M), 1,000 steps, dt 0.1 s."""
    rng = rng_for(1)
    sc = make_scene([per_lane] * n_lanes, rng)
    sc.update(K=K, dt=0.1, obs_stride=1, name="%dx%d K=%d" % (n_lanes, per_lane, K))
    return sc


def config2_tables(n_scen=4096, rng=None):
    """Uneven scenarios: lanes U[1,64], vehicles per lane U[2,200], horizons
    U[50,500], targets observed every 10th step."""
    rng = rng if rng is not None else rng_for(2)
    n_lanes = rng.integers(1, 65, size=n_scen)
    K = rng.integers(50, 501, size=n_scen)
    counts = [rng.integers(2, 201, size=int(L)) for L in n_lanes]
    return n_lanes, K, counts


def make_batch(lanes_per_scen, counts_per_scen, K, obs_stride, rng, dt=0.1):
    """Uneven scenarios laid out one after another: scenario s owns
    lanes_per_scen[s] lanes with the vehicle counts counts_per_scen[s], its
    own horizon K[s] and observation stride obs_stride[s]."""
    counts = np.concatenate([np.asarray(c, dtype=np.int64) for c in counts_per_scen])
    sc = make_scene(counts, rng)
    scen_lane_off = lane_offsets(lanes_per_scen)
    n_scen = len(lanes_per_scen)
    sc.update(scen_lane_off=scen_lane_off, K=np.asarray(K, dtype=np.int32),
              dt=np.full(n_scen, dt, dtype=np.float32), obs_stride=np.asarray(obs_stride, dtype=np.int32))
    lo = sc["lane_off"]
    sc["veh_off"] = lo[scen_lane_off]
    return sc


def config2(n_scen=4096):
    """4,096 scenarios: lanes U[1,64], vehicles per lane U[2,200], horizons
    U[50,500], dt 0.1 s, targets observed every 10th step."""
    rng = rng_for(2)
    n_lanes, K, counts = config2_tables(n_scen, rng)
    sc = make_batch(n_lanes, counts, K, np.full(n_scen, 10), rng)
    sc["name"] = "%d scenarios (%d lanes, %d vehicles), K U[50,500], obs every 10th step" % (
        n_scen, int(sc["scen_lane_off"][-1]), int(sc["lane_off"][-1]))
    return sc


def unsorted_view(sc, rng):
    """The same vehicles in a random order, with lane ids, as a layout step
    would receive them."""
    lane_off = sc["lane_off"]
    N = int(lane_off[-1])
    lane_id = np.repeat(np.arange(len(lane_off) - 1, dtype=np.int32), np.diff(lane_off))
    order = rng.permutation(N)
    return dict(lane_id=lane_id[order], p_init=sc["p_init"][order], order=order)


# ---------------------------------------------------------------------------
# Learned initializer (no counterpart in the paper)
# ---------------------------------------------------------------------------

# (fan_in, fan_out) of the four layers 80 -> 256 -> 256 -> 256 -> 5.
MLP_SIZES = ((80, 256), (256, 256), (256, 256), (256, 5))


def mlp_init(seed=0):
    """Flat initial weights (float32-exact float64), in the order W1, b1, ...,
    W4, b4 with W stored row = output unit: every entry uniform in
    [-1/sqrt(fan_in), 1/sqrt(fan_in)]."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 3 + 1000 * seed))
    parts = []
    for fan_in, fan_out in MLP_SIZES:
        bound = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=fan_out * fan_in))
        parts.append(rng.uniform(-bound, bound, size=fan_out))
    return f32(np.concatenate(parts))


def config3_train(n_lanes=100000, per_lane=100, K=20, seed=0):
    """Training scenes of the initializer: 100,000 lanes x 100 vehicles (10M
    samples) with the config-0 parameter and state ranges, simulated for the
    20-step observed prefix."""
    rng = rng_for(3, salt=1 + seed)
    sc = make_scene([per_lane] * n_lanes, rng)
    sc.update(K=K, dt=0.1, obs_stride=1, name="%dx%d K=%d (initializer training)" % (n_lanes, per_lane, K))
    return sc


def config3_fit(n_lanes=2000, per_lane=100, K=100):
    """Fit scenes of the initializer experiment: 2,000 lanes x 100 vehicles
    (200K), 100 steps, every step observed."""
    rng = rng_for(3)
    sc = make_scene([per_lane] * n_lanes, rng)
    sc.update(K=K, dt=0.1, obs_stride=1, name="%dx%d K=%d" % (n_lanes, per_lane, K))
    return sc


# ---- observed trajectories for the filtering / reconstruction mode ----------
#
# Stand-ins for the paper's trajectory data (Sec. V-B): NGSIM US-101 for
# filtering (6,101 trajectories, a position every 0.1 s, simulated with dt =
# 0.1 s) and a non-public Singapore set for reconstruction (21,750
# trajectories, sampling intervals of at least 1 s, up to 20 minutes long,
# dt = 1 s).  A trajectory is a smooth speed profile v(t) = vm + A1 sin(w1 t
# + f1) + A2 sin(w2 t + f2) with vm U[8, 25] m/s, A1 U[0, 0.3 vm], A2 U[0,
# 0.2 vm] (so v >= vm / 2 > 0), periods U[60, 300] s and U[15, 60] s; its
# closed-form position from a start U[0, 1000] m is sampled at the
# observation times and Gaussian noise is added.  Trajectories are returned
# longest first, so that neighbouring trajectories have similar horizons.

FILTER_SPEC = dict(n=6101, dur=(30.0, 90.0), dense=0.1, noise=0.3, dt=0.1)
RECON_SPEC = dict(n=21750, dur=(120.0, 1200.0), gap_min=1.0, gap_mean_extra=1.0, noise=1.0, dt=1.0)


def recon_observations(n, dur, rng, dense=None, gap_min=1.0, gap_mean_extra=1.0, noise=0.5, sort=True):
    """(obs_off int32 [n+1], obs_t, obs_p float32-exact float64 [n_obs]).
    dense: fixed sampling interval (s); else intervals gap_min + Exp(mean
    gap_mean_extra).  Timestamps start at 0 for every trajectory."""
    T = rng.uniform(dur[0], dur[1], size=n)
    if sort:
        T = np.sort(T)[::-1]
    vm = rng.uniform(8.0, 25.0, size=n)
    A1 = rng.uniform(0.0, 0.3, size=n) * vm
    A2 = rng.uniform(0.0, 0.2, size=n) * vm
    w1 = 2 * np.pi / rng.uniform(60.0, 300.0, size=n)
    w2 = 2 * np.pi / rng.uniform(15.0, 60.0, size=n)
    f1 = rng.uniform(0, 2 * np.pi, size=n)
    f2 = rng.uniform(0, 2 * np.pi, size=n)
    p0 = rng.uniform(0.0, 1000.0, size=n)
    ts = []
    for i in range(n):
        if dense is not None:
            t = np.arange(0.0, T[i] + 1e-9, dense)
        else:
            m = int(T[i] / gap_min) + 2
            t = np.concatenate([[0.0], np.cumsum(gap_min + rng.exponential(gap_mean_extra, size=m))])
            t = t[t <= T[i]]
        ts.append(f32(t))
    counts = np.array([len(t) for t in ts], dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.int32)
    off[1:] = np.cumsum(counts)
    t = np.concatenate(ts)
    idx = np.repeat(np.arange(n), counts)
    pos = (p0[idx] + vm[idx] * t - A1[idx] / w1[idx] * (np.cos(w1[idx] * t + f1[idx]) - np.cos(f1[idx]))
           - A2[idx] / w2[idx] * (np.cos(w2[idx] * t + f2[idx]) - np.cos(f2[idx])))
    pos = pos + rng.normal(0.0, noise, size=pos.shape)
    return off, t, f32(pos)


# ---- scenes for training-free prediction with lane geometry ----------------
#
# Stand-in for the Waymo Open Motion validation set (Sec. V-C): scenarios of
# U[2, 8] lane centre lines, each a circular arc (signed curvature of radius
# U[60, 1000] m) or, with probability 0.3, a straight line, 300 m long,
# starting at a point U[0, 200]^2 m with heading U[0, 2 pi), sampled every
# 2 m.  Every lane carries U[1, 6] agents, the first at arc length U[40, 70] m,
# each follower U[12, 25] m behind its predecessor; an agent moves along its
# lane with s(t) = s0 + vm t + (A / w)(cos f - cos(w t + f)) (vm U[3, 15] m/s
# per lane times U[0.9, 1.1] per agent, A U[0, 0.3 vm], period U[4, 12] s)
# at a lateral offset d0 + 0.2 sin(w2 t + f2) (d0 N(0, 0.4^2) m) plus
# position noise N(0, 0.1^2) m per coordinate.  Frames every 0.1 s: 11 of
# history (1 s) and 80 of future (8 s).  Positions on a lane come from the
# closed form of the arc, not from its polyline.

def prediction_scenes(n_scen, rng, n_hist=11, n_fut=80, dt=0.1, spacing=2.0, lane_len=300.0):
    F = n_hist + n_fut
    t = np.arange(F) * dt
    s_grid = np.arange(0.0, lane_len + 1e-9, spacing)
    M = len(s_grid)
    n_l = rng.integers(2, 9, size=n_scen)
    L = int(n_l.sum())
    scen_lane_off = np.zeros(n_scen + 1, np.int32)
    scen_lane_off[1:] = np.cumsum(n_l)
    x0, y0 = rng.uniform(0.0, 200.0, size=L), rng.uniform(0.0, 200.0, size=L)
    h0 = rng.uniform(0.0, 2 * np.pi, size=L)
    straight = rng.random(L) < 0.3
    k = np.where(straight, 0.0, rng.choice([-1.0, 1.0], size=L) / rng.uniform(60.0, 1000.0, size=L))

    def arc(l, s):
        """Point and heading at arc length s (broadcast) of lanes l."""
        kk, hh, xx, yy = k[l], h0[l], x0[l], y0[l]
        ks = np.where(kk == 0.0, 1.0, kk)
        h = hh + kk * s
        xc = np.where(kk == 0.0, xx + s * np.cos(hh), xx + (np.sin(h) - np.sin(hh)) / ks)
        yc = np.where(kk == 0.0, yy + s * np.sin(hh), yy - (np.cos(h) - np.cos(hh)) / ks)
        return xc, yc, h

    lanes = np.arange(L)
    px, py, _ = arc(lanes[:, None], s_grid[None, :])
    n_a = rng.integers(1, 7, size=L)
    A_n = int(n_a.sum())
    lane_of = np.repeat(lanes, n_a)
    first = np.repeat(np.cumsum(n_a) - n_a, n_a)
    rank = np.arange(A_n) - first                       # 0 = the lane's first agent
    gaps = np.where(rank == 0, 0.0, rng.uniform(12.0, 25.0, size=A_n))
    csum = np.cumsum(gaps)
    s0 = np.repeat(rng.uniform(40.0, 70.0, size=L), n_a) - (csum - csum[first])
    vm = np.repeat(rng.uniform(3.0, 15.0, size=L), n_a) * rng.uniform(0.9, 1.1, size=A_n)
    A = rng.uniform(0.0, 0.3, size=A_n) * vm
    w = 2 * np.pi / rng.uniform(4.0, 12.0, size=A_n)
    f = rng.uniform(0, 2 * np.pi, size=A_n)
    s = s0[None, :] + vm[None, :] * t[:, None] + (A / w)[None, :] * (np.cos(f)[None, :] - np.cos(w[None, :] * t[:, None] + f[None, :]))
    d = rng.normal(0.0, 0.4, size=A_n)[None, :] + 0.2 * np.sin(
        (2 * np.pi / rng.uniform(3.0, 9.0, size=A_n))[None, :] * t[:, None] + rng.uniform(0, 6.3, size=A_n)[None, :])
    cx, cy, h = arc(lane_of[None, :], s)
    x = cx - d * np.sin(h) + rng.normal(0.0, 0.1, size=(F, A_n))
    y = cy + d * np.cos(h) + rng.normal(0.0, 0.1, size=(F, A_n))
    scen_of = np.repeat(np.repeat(np.arange(n_scen), n_l), n_a)
    pt_off = (np.arange(L + 1) * M).astype(np.int32)
    return dict(pt_off=pt_off, px=f32(px.ravel()), py=f32(py.ravel()), x=f32(x), y=f32(y),
                lane_true=lane_of.astype(np.int32), lane_lo=scen_lane_off[scen_of], lane_hi=scen_lane_off[scen_of + 1],
                n_hist=n_hist, n_fut=n_fut, dt=float(np.float32(dt)), n_lanes=L)
