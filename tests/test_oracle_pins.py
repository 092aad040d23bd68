"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test pins the oracle to something other than itself: closed-form fixed
points of the modified model, invariants stated in Sec. III-C, a textbook
property of the IDM (intelligent braking), a dimensional-scaling invariance,
finite differences, an independent autograd differentiation, and library
routines (numpy logaddexp / lexsort, torch.optim.Adam).
"""
import numpy as np
import pytest

import oracle
from paper_2412_16750_gb300 import synth

A_MIN = -10.0


def lone_lanes(n):
    return np.arange(n + 1, dtype=np.int32)


def theta_of(v0, T, s0, am, b, delta):
    return np.stack([np.broadcast_to(np.asarray(x, dtype=np.float64), np.shape(v0)) for x in
                     (v0, T, s0, am, b, delta)]).astype(np.float64)


def eps_fixed(a_lb):
    """a at which the bounded acceleration a* vanishes: sp(a - a_lb) = -a_lb."""
    return np.log1p(-np.exp(a_lb))


# ---------------------------------------------------------------------------
# Free road (Eq. 2 with no interaction term, Sec. III-C bound, Eq. 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("delta", [4.0, 2.0, 3.5])
def test_free_road_fixed_point(delta):
    rng = np.random.default_rng(1)
    n = 40
    v0 = rng.uniform(25, 30, n)
    am = rng.uniform(1.5, 2.0, n)
    v_init = np.concatenate([rng.uniform(5, 20, n // 2), rng.uniform(35, 45, n - n // 2)])
    th = theta_of(v0, 1.5, 2.0, am, 2.0, delta)
    K, dt = 2500, 0.1
    P, V = oracle.forward(lone_lanes(n), np.full(n, 5.0), th, np.zeros(n), v_init, K, dt, A_MIN)
    eps = eps_fixed(A_MIN)  # v* > 1 m/s, so a_lb = a_min
    v_star = v0 * (1.0 - eps / am) ** (1.0 / delta)
    assert np.all(v_star > v0)  # the softplus bound lifts the fixed point above v0
    np.testing.assert_allclose(V[-1], v_star, rtol=0, atol=1e-9)
    # the approach is monotone
    d = np.diff(V, axis=0)
    below = v_init < v0
    assert np.all(d[:, below] >= -1e-12) and np.all(d[:, ~below] <= 1e-12)


def test_free_road_linear_decay_rate():
    """Near v*, the error shrinks per step by 1 + dt * da*/dv at v*, with
    da*/dv = sigma(eps - a_min) * (-a_max delta r*^(delta-1) / v0)."""
    v0, am, delta, dt = 30.0, 1.2, 4.0, 0.1
    th = theta_of(np.array([v0]), 1.5, 2.0, am, 2.0, delta)
    P, V = oracle.forward(lone_lanes(1), [5.0], th, [0.0], [29.0], 1500, dt, A_MIN)
    eps = eps_fixed(A_MIN)
    v_star = v0 * (1 - eps / am) ** (1 / delta)
    r = v_star / v0
    sig2 = 1.0 / (1.0 + np.exp(-(eps - A_MIN)))
    rate = 1.0 + dt * sig2 * (-am * delta * r ** (delta - 1) / v0)
    err = V[:, 0] - v_star
    ks = [k for k in range(len(err) - 1) if 1e-7 < abs(err[k]) < 1e-5]
    assert len(ks) > 10
    ratios = err[np.array(ks) + 1] / err[ks]
    np.testing.assert_allclose(ratios, rate, rtol=2e-6)


def test_vehicle_at_rest_creeps():
    """At v = 0: a_lb = max(-0/dt, a_min) = 0, so a* = sp(a_max) -- a creep,
    and a counterexample to the upper bound a* <= a_max claimed in Sec. III-C."""
    am = np.array([0.8, 1.0, 2.0, 7.5])
    n = len(am)
    th = theta_of(np.full(n, 30.0), 1.5, 2.0, am, 2.0, 4.0)
    dt = 0.1
    P, V, A = oracle.forward(lone_lanes(n), np.full(n, 5.0), th, np.zeros(n), np.zeros(n), 1, dt,
                             A_MIN, want_accel=True)
    np.testing.assert_allclose(A[0], np.logaddexp(0.0, am), rtol=1e-15)
    np.testing.assert_allclose(V[1], dt * np.logaddexp(0.0, am), rtol=1e-15)
    assert np.all(A[0] > am)
    np.testing.assert_array_equal(P[1], 0.0)  # position uses the old speed (Eq. 3)


# ---------------------------------------------------------------------------
# Steady platoon: the equilibrium gap of the modified model
# ---------------------------------------------------------------------------

def platoon(v, n, rng, small_s0=False):
    am = rng.uniform(0.8, 2.0, n)
    b = rng.uniform(1.0, 3.0, n)
    T = rng.uniform(1.0, 2.0, n)
    s0 = rng.uniform(0.2, 0.8, n) if small_s0 else rng.uniform(1.5, 3.0, n)
    delta = np.full(n, 4.0)
    v0 = v + rng.uniform(3.0, 10.0, n)
    dt = 0.1
    a_lb = max(-v / dt, A_MIN)
    eps = eps_fixed(a_lb)
    # head: free road with its fixed point at exactly v
    v0[0] = v / (1.0 - eps / am[0]) ** (1.0 / delta[0])
    length = rng.uniform(4.0, 6.0, n)
    sstar = np.logaddexp(0.0, s0 + v * T)  # sp(s_opt) at dv = 0
    gap = np.zeros(n)
    gap[1:] = sstar[1:] / np.sqrt(1.0 - (v / v0[1:]) ** delta[1:] - eps / am[1:])
    p = np.zeros(n)
    for i in range(1, n):
        p[i] = p[i - 1] - length[i - 1] - gap[i]
    th = np.stack([v0, T, s0, am, b, delta])
    return th, length, p, gap, dt


@pytest.mark.parametrize("v,small_s0", [(20.0, False), (8.0, False), (0.5, True)])
def test_steady_platoon(v, small_s0):
    rng = np.random.default_rng(7)
    n = 6
    th, length, p, gap, dt = platoon(v, n, rng, small_s0)
    K = 1000
    P, V = oracle.forward(np.array([0, n], dtype=np.int32), length, th, p, np.full(n, v), K, dt, A_MIN)
    np.testing.assert_allclose(V, v, rtol=0, atol=1e-9)
    gaps = P[:, :-1] - P[:, 1:] - length[:-1]
    np.testing.assert_allclose(gaps, np.broadcast_to(gap[1:], gaps.shape), rtol=0, atol=1e-9)
    np.testing.assert_allclose(P[-1] - P[0], K * dt * v, rtol=1e-12)


def test_platoon_uses_leader_length():
    """The gap subtracts the LEADER's length (Sec. III-A): swapping in the
    follower's own length breaks the equilibrium."""
    rng = np.random.default_rng(8)
    n = 4
    th, length, p, gap, dt = platoon(15.0, n, rng)
    length = np.array([4.0, 6.0, 4.5, 5.5])
    p = np.zeros(n)
    for i in range(1, n):
        p[i] = p[i - 1] - length[i - 1] - gap[i]
    P, V = oracle.forward(np.array([0, n], dtype=np.int32), length, th, p, np.full(n, 15.0), 50, dt, A_MIN)
    np.testing.assert_allclose(V, 15.0, atol=1e-10)


# ---------------------------------------------------------------------------
# Intelligent braking (textbook IDM property) pins Eq. 1's dv term
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kappa", [0.5, 1.0, 2.0])
def test_intelligent_braking(kappa):
    """With s0 = T = 0 and v0 -> inf, approaching a stopped leader at speed v
    and gap s, the IDM interaction term equals b_kin^2 / b with the kinematic
    deceleration b_kin = v^2 / (2 s): a = a_max - b_kin^2 / b."""
    v, am, b, dt = 20.0, 1.0, 2.0, 0.1
    b_kin = kappa * b
    s = v * v / (2.0 * b_kin)
    length = np.array([5.0, 5.0])
    th = np.array([[1e8, 1e8], [0.0, 0.0], [0.0, 0.0], [am, am], [b, b], [4.0, 4.0]])
    p = np.array([0.0, -(s + 5.0)])
    P, V, A = oracle.forward(np.array([0, 2], dtype=np.int32), length, th, p, np.array([0.0, v]), 1,
                             dt, A_MIN, want_accel=True)
    a_idm = am - b_kin ** 2 / b
    a_star = A_MIN + np.logaddexp(0.0, a_idm - A_MIN)
    np.testing.assert_allclose(A[0, 1], a_star, rtol=1e-12)


# ---------------------------------------------------------------------------
# Invariants of Sec. III-C
# ---------------------------------------------------------------------------

def test_positivity_and_lower_bound():
    rng = np.random.default_rng(3)
    sc = synth.make_scene([30] * 8, rng)
    # hard case: shrink gaps to a few metres and slow the leaders down
    p = sc["p_init"].copy()
    lane_off = sc["lane_off"]
    v = sc["v_init"].copy()
    for l in range(len(lane_off) - 1):
        a, e = lane_off[l], lane_off[l + 1]
        p[a:e] = -np.arange(e - a) * (5.0 + rng.uniform(1.0, 4.0))
        v[a] = 0.0
    P, V, A = oracle.forward(lane_off, sc["length"], sc["theta_true"], p, v, 300, 0.1, A_MIN, want_accel=True)
    # Sec. III-C guarantees non-negative speeds (strictly positive in exact
    # arithmetic; in floating point sp(a - a_lb) can underflow to 0 in a jam)
    assert np.all(V >= 0.0)
    assert (V[1:] == 0.0).any()  # the case really brakes to a stop
    assert np.all(A >= A_MIN)
    a_lb = np.maximum(-V[:-1] / 0.1, A_MIN)
    assert np.all(A >= a_lb)


def test_monotone_responses():
    """One step of a 2-vehicle lane: a* rises with the gap and with the
    leader's speed, and falls with the follower's own speed."""
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(50):
        th = synth.f32(np.array([[rng.uniform(25, 35)] * 2, [rng.uniform(1, 2)] * 2, [rng.uniform(1.5, 3)] * 2,
                                 [rng.uniform(0.8, 2)] * 2, [rng.uniform(1, 3)] * 2, [4.0, 4.0]]))
        gap = rng.uniform(10, 40)
        vf = rng.uniform(5, 25)
        vh = vf + rng.uniform(-5.0, 1.0)  # keeps s_opt > 0, where the interaction term acts

        def acc(gap, vf, vh):
            p = np.array([0.0, -(gap + 5.0)])
            _, _, A = oracle.forward(np.array([0, 2], dtype=np.int32), [5.0, 5.0], th, p,
                                     np.array([vh, vf]), 1, 0.1, A_MIN, want_accel=True)
            return A[0, 1]

        a0 = acc(gap, vf, vh)
        if a0 < A_MIN + 0.5:
            continue  # saturated at the lower bound: a* no longer moves
        checked += 1
        assert acc(gap + 0.5, vf, vh) > a0
        assert acc(gap, vf, vh + 0.5) > a0
        assert acc(gap, vf + 0.5, vh) < a0
    assert checked > 30


def test_scaling_invariance_textbook_limit():
    """With both softplus bounds inactive (s_opt >= ~40 m, a_min far below),
    the model is the textbook IDM with Euler steps, which is invariant under
    scaling every length by lam (positions, lengths, s0, speeds, v0, a_max, b)."""
    rng = np.random.default_rng(5)
    n_l, per = 3, 5
    N = n_l * per
    lane_off = synth.lane_offsets([per] * n_l)
    length = np.full(N, 5.0)
    gaps = rng.uniform(60.0, 100.0, N)
    p = np.zeros(N)
    for l in range(n_l):
        for i in range(lane_off[l] + 1, lane_off[l + 1]):
            p[i] = p[i - 1] - length[i - 1] - gaps[i]
    v = rng.uniform(24.0, 26.0, N)
    th = np.stack([rng.uniform(28, 35, N), rng.uniform(1.8, 2.5, N), rng.uniform(1.5, 3, N),
                   rng.uniform(1.0, 2.0, N), rng.uniform(1.0, 3.0, N), np.full(N, 4.0)])
    lam = 2.0
    kw = dict(K=80, dt=0.1, a_min=-1e4)
    P1, V1 = oracle.forward(lane_off, length, th, p, v, **kw)
    th2 = th.copy()
    th2[[0, 2, 3, 4]] *= lam
    P2, V2 = oracle.forward(lane_off, lam * length, th2, lam * p, lam * v, **kw)
    np.testing.assert_allclose(P2, lam * P1, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(V2, lam * V1, rtol=1e-12)


def test_lane_order_equivariance():
    rng = np.random.default_rng(6)
    counts = [3, 7, 1, 5]
    sc = synth.make_scene(counts, rng)
    K, dt = 40, 0.1
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, dt)
    order = [2, 0, 3, 1]
    lo = sc["lane_off"]
    idx = np.concatenate([np.arange(lo[l], lo[l + 1]) for l in order])
    lane_off2 = synth.lane_offsets([counts[l] for l in order])
    P2, V2 = oracle.forward(lane_off2, sc["length"][idx], sc["theta_true"][:, idx], sc["p_init"][idx],
                            sc["v_init"][idx], K, dt)
    np.testing.assert_array_equal(P2, P[:, idx])
    np.testing.assert_array_equal(V2, V[:, idx])


# ---------------------------------------------------------------------------
# Loss
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("stride", [1, 3, 7])
def test_loss_constant_offset(stride):
    """targets = P + c at every observed step gives L = N c^2 exactly."""
    rng = np.random.default_rng(9)
    K, N = 20, 6
    P = rng.normal(size=(K + 1, N)) * 100
    c = 0.75
    n_obs = K // stride
    Y = P[stride::stride][:n_obs] + c
    L, gP = oracle.mse_seed(P, Y, stride)
    assert L == pytest.approx(N * c * c, rel=1e-12)
    obs = np.zeros(K + 1, dtype=bool)
    obs[stride::stride] = True
    obs[(n_obs + 1) * stride:] = False
    np.testing.assert_allclose(gP[obs], -2.0 * c / n_obs, rtol=1e-12)
    assert np.all(gP[~obs] == 0.0)


def test_loss_stride_beyond_horizon():
    P = np.ones((6, 3))
    L, gP = oracle.mse_seed(P, np.zeros((0, 3)), 10)
    assert L == 0.0 and np.all(gP == 0.0)


# ---------------------------------------------------------------------------
# Gradients: finite differences, independent autograd, zero residual
# ---------------------------------------------------------------------------

def tiny_problem(seed=11, counts=(3, 3), K=20, stride=1, near_truth=False):
    rng = np.random.default_rng(seed)
    sc = synth.make_scene(list(counts), rng)
    N = int(sc["lane_off"][-1])
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, 0.1)
    n_obs = K // stride
    Y = P[stride::stride][:n_obs] + rng.normal(0, 0.5, size=(n_obs, N))
    th = sc["theta_true"] * (1 + rng.uniform(-0.1, 0.1, size=(6, N))) if near_truth else \
        sc["theta_true"] * rng.uniform(0.7, 1.3, size=(6, N))
    th[5] = rng.uniform(3.0, 5.0, N)
    return sc, th, Y, K, stride


def loss_of(sc, th, Y, K, stride, p_init=None, v_init=None):
    P, V = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"] if p_init is None else p_init,
                          sc["v_init"] if v_init is None else v_init, K, 0.1)
    return oracle.mse_seed(P, Y, stride)[0]


@pytest.mark.parametrize("stride,near", [(1, False), (4, True)])
def test_adjoint_matches_central_differences(stride, near):
    sc, th, Y, K, s = tiny_problem(stride=stride, near_truth=near)
    P, V = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, 0.1)
    assert np.all(V > 1.05)  # away from the a_lb kink at v = -a_min dt
    L, gP = oracle.mse_seed(P, Y, s)
    gth, gp0, gv0 = oracle.adjoint(sc["lane_off"], sc["length"], th, K, 0.1, P, V, gP)
    N = th.shape[1]
    fd = np.zeros((6, N))
    for q in range(6):
        for i in range(N):
            h = 1e-6 * max(1.0, abs(th[q, i]))
            tp, tm = th.copy(), th.copy()
            tp[q, i] += h
            tm[q, i] -= h
            fd[q, i] = (loss_of(sc, tp, Y, K, s) - loss_of(sc, tm, Y, K, s)) / (2 * h)
    for q in range(6):
        np.testing.assert_allclose(gth[q], fd[q], rtol=1e-5, atol=1e-7 * np.abs(fd[q]).max())
    for arr, name in ((gp0, "p"), (gv0, "v")):
        fdx = np.zeros(N)
        for i in range(N):
            h = 1e-6
            xp = sc[name + "_init"].copy()
            xm = xp.copy()
            xp[i] += h
            xm[i] -= h
            kw_p = {name + "_init": xp}
            kw_m = {name + "_init": xm}
            fdx[i] = (loss_of(sc, th, Y, K, s, **kw_p) - loss_of(sc, th, Y, K, s, **kw_m)) / (2 * h)
        np.testing.assert_allclose(arr, fdx, rtol=1e-5, atol=1e-7 * np.abs(fdx).max())


def test_adjoint_matches_torch_autograd():
    """A separate vectorised restatement of Eq. 1-3 and the Sec. III-C bounds,
    differentiated by torch autograd in float64 (the paper's own approach)."""
    torch = pytest.importorskip("torch")
    sc, th, Y, K, s = tiny_problem(seed=12, counts=(4, 1, 3), K=30, stride=2)
    lane_off = sc["lane_off"]
    N = th.shape[1]
    has_leader = np.ones(N, dtype=bool)
    has_leader[lane_off[:-1]] = False
    lead = np.maximum(np.arange(N) - 1, 0)

    t = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    p = torch.tensor(sc["p_init"], dtype=torch.float64, requires_grad=True)
    v = torch.tensor(sc["v_init"], dtype=torch.float64, requires_grad=True)
    gV_seed = torch.tensor(np.random.default_rng(2).normal(size=(K + 1, N)) * 1e-3)
    hl = torch.tensor(has_leader)
    ld = torch.tensor(lead)
    ln = torch.tensor(sc["length"], dtype=torch.float64)
    dt = 0.1
    pk, vk = p, v
    Ps, Vs = [pk], [vk]
    v0_, T_, s0_, am_, b_, dl_ = t
    for k in range(K):
        gap = torch.where(hl, pk[ld] - pk - ln[ld], torch.full_like(pk, 1e9))
        gap = torch.clamp(gap, min=0.1)
        dv = vk - vk[ld]
        s_opt = s0_ + vk * T_ + vk * dv / (2 * torch.sqrt(am_ * b_))
        z = torch.where(hl, torch.nn.functional.softplus(s_opt) / gap, torch.zeros_like(pk))
        a = am_ * (1 - (vk / v0_) ** dl_ - z ** 2)
        a_lb = torch.maximum(-vk / dt, torch.full_like(vk, A_MIN))
        a_star = a_lb + torch.nn.functional.softplus(a - a_lb)
        pk, vk = pk + dt * vk, vk + dt * a_star
        Ps.append(pk)
        Vs.append(vk)
    Pt = torch.stack(Ps)
    Vt = torch.stack(Vs)
    n_obs = K // s
    Yt = torch.tensor(Y)
    L = (((Pt[s::s][:n_obs] - Yt) ** 2).mean(dim=0)).sum() + (Vt * gV_seed).sum()
    L.backward()

    P, V = oracle.forward(lane_off, sc["length"], th, sc["p_init"], sc["v_init"], K, dt)
    np.testing.assert_allclose(P, Pt.detach().numpy(), rtol=0, atol=1e-9)
    Lo, gP = oracle.mse_seed(P, Y, s)
    gth, gp0, gv0 = oracle.adjoint(lane_off, sc["length"], th, K, dt, P, V, gP, gV_seed.numpy())
    np.testing.assert_allclose(gth, t.grad.numpy(), rtol=1e-8, atol=1e-10 * np.abs(t.grad.numpy()).max())
    np.testing.assert_allclose(gp0, p.grad.numpy(), rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(gv0, v.grad.numpy(), rtol=1e-8, atol=1e-12)


def test_zero_residual_gives_zero_gradient():
    sc, _, _, K, s = tiny_problem(seed=13)
    th = sc["theta_true"]
    P, V = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, 0.1)
    L, gP = oracle.mse_seed(P, P[1:], 1)
    assert L == 0.0
    gth, gp0, gv0 = oracle.adjoint(sc["lane_off"], sc["length"], th, K, 0.1, P, V, gP)
    assert np.all(gth == 0.0) and np.all(gp0 == 0.0) and np.all(gv0 == 0.0)


# ---------------------------------------------------------------------------
# Adam + projection, fit, layout
# ---------------------------------------------------------------------------

def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(14)
    N = 17
    th = rng.uniform(1, 9, size=(5, N))
    lo = np.array([2.0, 1.5, 1.0, 3.0, 2.5])
    hi = np.array([8.0, 8.5, 7.0, 9.0, 6.0])
    th = np.clip(th, lo[:, None], hi[:, None])
    m = np.zeros((5, N))
    v = np.zeros((5, N))
    tt = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.Adam([tt], lr=0.1, betas=(0.9, 0.999), eps=1e-8)
    n_iter = 6
    for it in range(n_iter):
        g = rng.normal(size=(5, N)) * 10 ** rng.uniform(-3, 1)
        lr = oracle.lr_schedule(it, n_iter, 0.1, 0.01)
        oracle.adam_step(th, g, m, v, it + 1, lr, lo, hi)
        for grp in opt.param_groups:
            grp["lr"] = lr
        tt.grad = torch.tensor(g)
        opt.step()
        with torch.no_grad():
            tt.copy_(torch.maximum(torch.minimum(tt, torch.tensor(hi)[:, None]), torch.tensor(lo)[:, None]))
        np.testing.assert_allclose(th, tt.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert oracle.lr_schedule(0, 5, 0.1, 0.01) == 0.1
    assert oracle.lr_schedule(4, 5, 0.1, 0.01) == pytest.approx(0.01, abs=1e-17)


def test_fit_is_the_replay_of_its_steps():
    """oracle.fit = n_iter rounds of (forward, squared-error seed, adjoint,
    Adam with bias correction at t = it + 1 and the learning rate
    lr0 + (lr1 - lr0) it / (n_iter - 1) written here from its definition,
    projection onto the box), with the loss recorded before each update and
    delta never changed."""
    sc = synth.make_scene([6, 3, 9], np.random.default_rng(19))
    K, s, n_iter, lr0, lr1 = 24, 2, 4, 0.3, 0.05
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, 0.1)
    N = P.shape[1]
    Y = P[s::s][:K // s] + np.random.default_rng(20).normal(0, 0.5, size=(K // s, N))
    th0 = synth.plain_init(N)
    th0[5, :3] = 3.0
    lo, hi = np.array(synth.BOX_LO), np.array(synth.BOX_HI)
    thf, hist = oracle.fit(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K, 0.1, Y, s, n_iter,
                           lr0, lr1, lo, hi)
    th = th0.copy()
    m, v = np.zeros((5, N)), np.zeros((5, N))
    for it in range(n_iter):
        Pi, Vi = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, 0.1)
        L, gP = oracle.mse_seed(Pi, Y, s)
        g, _, _ = oracle.adjoint(sc["lane_off"], sc["length"], th, K, 0.1, Pi, Vi, gP)
        assert hist[it] == pytest.approx(L, rel=1e-14)
        th5 = np.ascontiguousarray(th[:5])
        oracle.adam_step(th5, np.ascontiguousarray(g[:5]), m, v, it + 1, lr0 + (lr1 - lr0) * it / (n_iter - 1),
                         lo, hi)
        th[:5] = th5
    np.testing.assert_allclose(thf, th, rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(thf[5], th0[5])


def test_fit_from_truth_without_noise_is_stationary():
    sc, _, _, K, s = tiny_problem(seed=15)
    th = sc["theta_true"].copy()
    P, V = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, 0.1)
    thf, hist = oracle.fit(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, 0.1,
                           P[1:], 1, 3, 0.1, 0.01, synth.BOX_LO, synth.BOX_HI)
    assert np.all(hist == 0.0)
    np.testing.assert_array_equal(thf, th)


def test_fit_reduces_loss():
    sc = synth.make_scene([20] * 3, np.random.default_rng(16))
    K = 60
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, 0.1)
    Y = P[1:] + np.random.default_rng(17).normal(0, 0.5, size=(K, P.shape[1]))
    th0 = synth.plain_init(P.shape[1])
    thf, hist = oracle.fit(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K, 0.1,
                           Y, 1, 40, 0.1, 0.01, synth.BOX_LO, synth.BOX_HI)
    assert hist[-1] < 0.2 * hist[0]
    assert np.all(thf[5] == 4.0)
    assert np.all(thf[:5] >= np.array(synth.BOX_LO)[:, None]) and np.all(thf[:5] <= np.array(synth.BOX_HI)[:, None])


def test_layout_matches_lexsort():
    rng = np.random.default_rng(18)
    N, L = 500, 37
    lane = rng.integers(0, L, size=N).astype(np.int32)
    pos = synth.f32(rng.uniform(-100, 0, size=N))
    pos[::7] = pos[0]  # ties broken by original index
    perm, lane_off = oracle.layout(lane, pos, L)
    ref = np.lexsort((np.arange(N), -pos, lane))
    np.testing.assert_array_equal(perm, ref)
    np.testing.assert_array_equal(lane_off, np.concatenate([[0], np.cumsum(np.bincount(lane, minlength=L))]))


def test_layout_recovers_generated_order():
    sc = synth.config0()
    u = synth.unsorted_view(sc, np.random.default_rng(19))
    perm, lane_off = oracle.layout(u["lane_id"], u["p_init"], 10)
    np.testing.assert_array_equal(lane_off, sc["lane_off"])
    np.testing.assert_array_equal(u["order"][perm], np.arange(1000))


def test_gap_floor_reading():
    """Reading for gaps at or below zero (the paper is silent): the gap is
    floored at 0.1 m, so any raw gap below the floor acts like 0.1 m and its
    derivative is zero."""
    th = np.array([[30.0] * 2, [1.5] * 2, [2.0] * 2, [1.0] * 2, [2.0] * 2, [4.0] * 2])

    def step(raw_gap):
        p = np.array([0.0, -(raw_gap + 5.0)])
        _, _, A = oracle.forward(np.array([0, 2], dtype=np.int32), [5.0, 5.0], th, p,
                                 np.array([0.5, 0.5]), 1, 0.1, A_MIN, want_accel=True)
        return A[0, 1]

    a_floor = step(0.1)
    for g in (0.09, 0.0, -0.5, -3.0):
        assert step(g) == a_floor
    assert step(3.0) > a_floor  # the floor is a bound, not a constant
