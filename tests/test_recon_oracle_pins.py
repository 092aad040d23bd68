"""Pins of the FP64 single-trajectory reconstruction oracle (paper Sec. IV-A:
one ego vehicle per trajectory behind a virtual leader with per-step gap and
speed-difference variables, MAE at the nearest steps)."""
import math

import numpy as np
import pytest

import oracle
from oracle import recon as R
from paper_2412_16750_gb300 import synth

DT = 0.1
A_MIN = -10.0


def test_virtual_leader_reproduces_a_coupled_follower():
    # a real lane: the follower's gap and speed difference, fed to the
    # single-trajectory model, give back the follower's trajectory
    rng = np.random.default_rng(1)
    sc = synth.make_scene([3], rng)
    K = 200
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    for f in (1, 2):
        gap = P[:K, f - 1] - P[:K, f] - sc["length"][f - 1]
        dv = V[:K, f] - V[:K, f - 1]
        Pr, Vr, _ = R.forward([K], gap[:, None], dv[:, None], sc["theta_true"][:, f:f + 1], [sc["p_init"][f]],
                              [sc["v_init"][f]], DT, A_MIN)
        np.testing.assert_allclose(Pr[:, 0], P[:, f], rtol=0, atol=1e-9)
        np.testing.assert_allclose(Vr[:, 0], V[:, f], rtol=0, atol=1e-9)


def test_far_leader_is_free_road():
    th = np.array([[30.0], [1.5], [2.0], [1.2], [2.0], [4.0]])
    K = 2000
    Pr, Vr, _ = R.forward([K], np.full((K, 1), 1e7), np.zeros((K, 1)), th, [0.0], [12.0], DT, A_MIN)
    eps = math.log(1 - math.exp(A_MIN))
    v_star = 30.0 * (1 - eps / 1.2) ** 0.25
    assert abs(Vr[-1, 0] - v_star) < 1e-6


def test_nearest_step_brute_force():
    rng = np.random.default_rng(2)
    ks = np.arange(0, 600)
    for t in np.concatenate([rng.uniform(0, 50, 2000), np.arange(0, 5, 0.05)]):
        d = np.abs(t - ks * DT)
        order = np.argsort(d)
        if d[order[1]] - d[order[0]] < 1e-9:
            continue                                   # a half-step tie in decimal, rounding decides
        assert R.nearest_step(t, DT) == ks[order[0]], t
    # exact ties (binary step): the later step
    for j in range(40):
        assert R.nearest_step((j + 0.5) * 0.125, 0.125) == j + 1


def _toy(seed, N=3, Kmax=25):
    rng = np.random.default_rng(seed)
    K = rng.integers(15, Kmax + 1, size=N).astype(np.int32)
    th = np.vstack([rng.uniform(25, 35, N), rng.uniform(1, 2, N), rng.uniform(1.5, 3, N), rng.uniform(0.8, 2, N),
                    rng.uniform(1, 3, N), np.full(N, 4.0)])
    dp = rng.uniform(15, 40, (Kmax, N))
    dv = rng.uniform(-3, 3, (Kmax, N))
    p0, v0 = rng.uniform(-50, 0, N), rng.uniform(12, 25, N)
    # observations at random steps 1..K_i, shifted by +-(2..6) m so that the
    # signs of the residuals do not flip under small perturbations
    off, ks, ys = [0], [], []
    P, _, _ = R.forward(K, dp, dv, th, p0, v0, DT, A_MIN)
    for i in range(N):
        steps = np.sort(rng.choice(np.arange(1, K[i] + 1), size=6, replace=False))
        for k in steps:
            ks.append(k)
            ys.append(P[k, i] + rng.choice([-1, 1]) * rng.uniform(2, 6))
        off.append(len(ks))
    return K, th, dp, dv, p0, v0, np.array(off, np.int32), np.array(ks, np.int32), np.array(ys)


def _loss(K, th, dp, dv, p0, v0, off, ks, ys):
    P, _, _ = R.forward(K, dp, dv, th, p0, v0, DT, A_MIN)
    return R.mae_seed(K, off, ks, ys, P)[0]


def test_adjoint_matches_finite_differences():
    K, th, dp, dv, p0, v0, off, ks, ys = _toy(3)
    P, V, _ = R.forward(K, dp, dv, th, p0, v0, DT, A_MIN)
    L, gP = R.mae_seed(K, off, ks, ys, P)
    g, gdp, gdv, gp0, gv0 = R.adjoint(K, dp, dv, th, DT, V, gP, A_MIN)

    def fd(fun, x, h):
        return (fun(x + h) - fun(x - h)) / (2 * h)

    for i in range(3):
        for q in range(6):
            def f(x, q=q, i=i):
                t = th.copy(); t[q, i] = x
                return _loss(K, t, dp, dv, p0, v0, off, ks, ys)
            h = 1e-6 * max(1.0, abs(th[q, i]))
            assert abs(fd(f, th[q, i], h) - g[q, i]) <= 1e-5 * max(1.0, abs(g[q, i])), (q, i)
        for k in (0, 5, K[i] - 1):
            def fp(x, k=k, i=i):
                d = dp.copy(); d[k, i] = x
                return _loss(K, th, d, dv, p0, v0, off, ks, ys)

            def fv(x, k=k, i=i):
                d = dv.copy(); d[k, i] = x
                return _loss(K, th, dp, d, p0, v0, off, ks, ys)
            assert abs(fd(fp, dp[k, i], 1e-6) - gdp[k, i]) <= 1e-6 * max(1.0, abs(gdp[k, i]))
            assert abs(fd(fv, dv[k, i], 1e-6) - gdv[k, i]) <= 1e-6 * max(1.0, abs(gdv[k, i]))
        def f0(x, i=i):
            p = p0.copy(); p[i] = x
            return _loss(K, th, dp, dv, p, v0, off, ks, ys)

        def f1(x, i=i):
            v = v0.copy(); v[i] = x
            return _loss(K, th, dp, dv, p0, v, off, ks, ys)
        assert abs(fd(f0, p0[i], 1e-6) - gp0[i]) <= 1e-6 * max(1.0, abs(gp0[i]))
        assert abs(fd(f1, v0[i], 1e-6) - gv0[i]) <= 1e-6 * max(1.0, abs(gv0[i]))
    # entries beyond each trajectory's horizon carry no gradient
    for i in range(3):
        assert np.all(gdp[K[i]:, i] == 0) and np.all(gdv[K[i]:, i] == 0)


def test_adjoint_matches_autograd_restatement():
    torch = pytest.importorskip("torch")
    K, th, dp, dv, p0, v0, off, ks, ys = _toy(4, N=2)
    rng = np.random.default_rng(5)
    Kmax = dp.shape[0]
    P, V, _ = R.forward(K, dp, dv, th, p0, v0, DT, A_MIN)
    w = rng.normal(size=P.shape)                      # arbitrary dense seeds
    for i in range(2):
        w[K[i] + 1:, i] = 0.0
    w[0] = 0.0
    g, gdp, gdv, gp0, gv0 = R.adjoint(K, dp, dv, th, DT, V, w, A_MIN)
    sp = torch.nn.functional.softplus
    for i in range(2):
        t = torch.tensor(th[:, i], requires_grad=True)
        d1 = torch.tensor(dp[:, i], requires_grad=True)
        d2 = torch.tensor(dv[:, i], requires_grad=True)
        p = torch.tensor(p0[i], dtype=torch.float64, requires_grad=True)
        v = torch.tensor(v0[i], dtype=torch.float64, requires_grad=True)
        pk, vk, loss = p, v, 0.0
        for k in range(K[i]):
            c = 1 / (2 * torch.sqrt(t[3] * t[4]))
            s = sp(t[2] + vk * t[1] + vk * d2[k] * c)
            gap = torch.clamp(d1[k], min=0.1)
            a = t[3] * (1 - (vk / t[0]) ** t[5] - (s / gap) ** 2)
            lbv = -vk / DT
            alb = lbv if lbv.item() > A_MIN else torch.tensor(A_MIN, dtype=torch.float64)
            ast = alb + sp(a - alb)
            pk, vk = pk + DT * vk, vk + DT * ast
            loss = loss + float(w[k + 1, i]) * pk
        loss.backward()
        np.testing.assert_allclose(t.grad.numpy(), g[:, i], rtol=1e-7, atol=1e-10)
        np.testing.assert_allclose(d1.grad.numpy()[:K[i]], gdp[:K[i], i], rtol=1e-7, atol=1e-10)
        np.testing.assert_allclose(d2.grad.numpy()[:K[i]], gdv[:K[i], i], rtol=1e-7, atol=1e-10)
        assert abs(p.grad.item() - gp0[i]) < 1e-8 and abs(v.grad.item() - gv0[i]) < 1e-8


def test_mae_closed_form_and_zero_residual():
    K, th, dp, dv, p0, v0, off, ks, ys = _toy(6)
    P, _, _ = R.forward(K, dp, dv, th, p0, v0, DT, A_MIN)
    exact = np.array([P[k, i] for i in range(3) for k in ks[off[i]:off[i + 1]]])
    L, gP = R.mae_seed(K, off, ks, exact + 2.5, P)
    assert abs(L - 2.5 * len(ks)) < 1e-9
    assert np.all(gP[ks, np.repeat(np.arange(3), np.diff(off))] == -1.0)
    L0, g0 = R.mae_seed(K, off, ks, exact, P)
    assert L0 == 0.0 and np.all(g0 == 0.0)          # sign(0) = 0


def test_initial_state_rule():
    off = np.array([0, 3, 5], np.int32)
    t = np.array([0.0, 0.5, 1.0, 0.0, 2.0])
    y = np.array([10.0, 18.0, 25.0, -4.0, 36.0])
    p0, v0 = R.init_state(off, t, y)
    np.testing.assert_allclose(p0, [10.0, -4.0])
    np.testing.assert_allclose(v0, [16.0, 20.0])
    # a backwards first difference, equal timestamps and a single observation give 0
    p0, v0 = R.init_state(np.array([0, 2, 4, 5], np.int32), np.array([0.0, 1.0, 3.0, 3.0, 7.0]),
                          np.array([5.0, 4.0, 1.0, 2.0, 9.0]))
    np.testing.assert_array_equal(v0, [0.0, 0.0, 0.0])
    np.testing.assert_array_equal(p0, [5.0, 1.0, 9.0])


def test_fit_reduces_loss_and_is_stationary_at_the_truth():
    K, th, dp, dv, p0, v0, off, ks, ys = _toy(7)
    lo, hi = synth.BOX_LO, synth.BOX_HI
    th_f, dp_f, dv_f, hist = R.fit(K, np.full_like(dp, 10.0), np.zeros_like(dv), synth.plain_init(3), p0, v0, DT,
                                   off, ks, ys, 60, 0.1, 0.01, lo, hi, A_MIN)
    assert hist[-1] < 0.5 * hist[0]
    P, _, _ = R.forward(K, dp, dv, th, p0, v0, DT, A_MIN)
    exact = np.array([P[k, i] for i in range(3) for k in ks[off[i]:off[i + 1]]])
    th2, dp2, dv2, hist2 = R.fit(K, dp, dv, th, p0, v0, DT, off, ks, exact, 5, 0.1, 0.01, lo, hi, A_MIN)
    assert np.all(hist2 == 0.0)
    np.testing.assert_array_equal(dp2, dp)
    np.testing.assert_array_equal(th2[:5], np.clip(th[:5], np.array(lo)[:, None], np.array(hi)[:, None]))


def test_fit_is_the_replay_of_its_steps():
    """R.fit = n_iter rounds of (forward, absolute-error seed with the loss
    recorded before the update, adjoint, Adam at t = it + 1 with the learning
    rate lr0 + (lr1 - lr0) it / (n_iter - 1) on the five parameters, projected
    onto the box, and unconstrained on every dp_k, dv_k), replayed here with
    torch.optim.Adam; delta is never changed."""
    torch = pytest.importorskip("torch")
    K, th, dp, dv, p0, v0, off, ks, ys = _toy(21)
    dv[2:6, 0] = 25.0     # far outside any plausible bound: the virtual-leader
    dp[3:5, 1] = 400.0    # variables are never boxed
    lo, hi = np.array(synth.BOX_LO), np.array(synth.BOX_HI)
    th0 = synth.plain_init(3)
    th0[5, 1] = 3.0
    n_iter, lr0, lr1 = 5, 0.2, 0.02
    th_f, dp_f, dv_f, hist = R.fit(K, dp, dv, th0, p0, v0, DT, off, ks, ys, n_iter, lr0, lr1, lo, hi, A_MIN)
    t_th = torch.tensor(th0[:5].copy(), requires_grad=True)
    t_dp = torch.tensor(dp.copy(), requires_grad=True)
    t_dv = torch.tensor(dv.copy(), requires_grad=True)
    opt = torch.optim.Adam([t_th, t_dp, t_dv], lr=lr0, betas=(0.9, 0.999), eps=1e-8)
    for it in range(n_iter):
        thi = np.vstack([t_th.detach().numpy(), th0[5:]])
        dpi, dvi = t_dp.detach().numpy(), t_dv.detach().numpy()
        P, V, _ = R.forward(K, dpi, dvi, thi, p0, v0, DT, A_MIN)
        L, gP = R.mae_seed(K, off, ks, ys, P)
        g, gdp, gdv, _, _ = R.adjoint(K, dpi, dvi, thi, DT, V, gP, A_MIN)
        assert hist[it] == pytest.approx(L, rel=1e-14)
        for grp in opt.param_groups:
            grp["lr"] = lr0 + (lr1 - lr0) * it / (n_iter - 1)
        t_th.grad, t_dp.grad, t_dv.grad = torch.tensor(g[:5]), torch.tensor(gdp), torch.tensor(gdv)
        opt.step()
        with torch.no_grad():
            t_th.copy_(torch.maximum(torch.minimum(t_th, torch.tensor(hi)[:, None]), torch.tensor(lo)[:, None]))
    np.testing.assert_allclose(th_f[:5], t_th.detach().numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(th_f[5], th0[5])
    np.testing.assert_allclose(dp_f, t_dp.detach().numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dv_f, t_dv.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert not np.allclose(dp_f, dp)


def test_metrics_hand_made():
    K = np.array([4, 4], np.int32)
    P = np.array([[3.0, 0.0], [4.0, 2.0], [5.0, 4.0], [6.0, 6.0], [7.0, 8.0]])
    A = np.array([[1.0, -2.0], [5.0, 12.0], [-1.0, 2.0], [1.0, -2.0]])
    off = np.array([0, 2, 4], np.int32)
    ks = np.array([0, 4, 0, 4], np.int32)
    ys = np.array([3.0, 7.4, 0.0, 8.0])             # trajectory 0: error 0.4 at k=4 over length 4.4
    pos, mean, std, imp = R.metrics(K, off, ks, ys, P, A)
    assert abs(pos - (0.4 / 4.4) / 4) < 1e-12
    absa = np.abs(A).ravel()
    assert abs(mean - absa.mean()) < 1e-12 and abs(std - absa.std()) < 1e-12
    assert imp == 0.5                                # |a*| = 5 in trajectory 0 is not implausible


def test_mae_several_observations_per_step():
    # two observations at one step: both enter the loss, the seed is the sum
    # of their signs (here one on each side of the position: seed 0)
    K = np.array([3], np.int32)
    P = np.array([[0.0], [1.0], [2.0], [3.0]])
    off = np.array([0, 4], np.int32)
    ks = np.array([0, 2, 2, 3], np.int32)
    ys = np.array([0.0, 3.0, -1.0, 5.0])
    L, gP = R.mae_seed(K, off, ks, ys, P)
    assert L == 1.0 + 3.0 + 2.0
    np.testing.assert_array_equal(gP[:, 0], [0.0, 0.0, 0.0, -1.0])
    L, gP = R.mae_seed(K, off, np.array([0, 2, 2, 2], np.int32), np.array([0.0, 3.0, 4.0, -1.0]), P)
    assert L == 1.0 + 2.0 + 3.0 and gP[2, 0] == -1.0


def test_gap_floor_has_zero_derivative():
    # virtual-leader gaps below the floor: the loss does not depend on them
    K, th, dp, dv, p0, v0, off, ks, ys = _toy(9)
    dp = dp.copy()
    dp[2:6, :] = 0.05
    P, V, _ = R.forward(K, dp, dv, th, p0, v0, DT, A_MIN)
    _, gP = R.mae_seed(K, off, ks, ys, P)
    _, gdp, _, _, _ = R.adjoint(K, dp, dv, th, DT, V, gP, A_MIN)
    assert np.all(gdp[2:6, :] == 0.0)
    L0 = _loss(K, th, dp, dv, p0, v0, off, ks, ys)
    d2 = dp.copy()
    d2[3, 1] = 0.07
    assert _loss(K, th, d2, dv, p0, v0, off, ks, ys) == L0
    # the same steps with their original (above-floor) gaps do have a derivative
    K, th, dp0, dv, p0, v0, off, ks, ys = _toy(9)
    P, V, _ = R.forward(K, dp0, dv, th, p0, v0, DT, A_MIN)
    _, gP = R.mae_seed(K, off, ks, ys, P)
    _, gdp0, _, _, _ = R.adjoint(K, dp0, dv, th, DT, V, gP, A_MIN)
    assert np.any(gdp0[2:6, :] != 0.0)
