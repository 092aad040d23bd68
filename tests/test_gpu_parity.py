"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerances (the workload statement's bar):
  * positions: max |p_gpu - p_oracle| <= 1e-3 m over 100 steps;
  * gradients: for each of the six parameters, ||g_gpu - g_ref|| / ||g_ref||
    <= 1e-4, and every element within 1e-4 * max |g_ref|;
  * integer work (layout permutation): bit-exact.
Both sides start from identical float32-representable inputs (dt is the
float32 value of 0.1 on both sides).
"""
import numpy as np
import pytest

import oracle
from paper_2412_16750_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = float(np.float32(0.1))
A_MIN = -10.0
POS_TOL = 1e-3
GRAD_RTOL = 1e-4
GRAD_ELEM = 1e-4


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16750_gb300 import api as _api
    return _api


def cuda(x, dtype=None):
    dtype = dtype or torch.float32
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def scene_of(api, sc):
    return api.Scene.from_lane_off(cuda(sc["lane_off"], torch.int32), cuda(sc["length"]))


def grad_close(g, ref, rtol=GRAD_RTOL, elem=GRAD_ELEM, rows=range(6)):
    for q in rows:
        nr = np.linalg.norm(ref[q])
        if nr == 0.0:
            assert np.max(np.abs(g[q])) <= 1e-30 + 1e-6 * np.max(np.abs(ref)), q
            continue
        err = np.linalg.norm(g[q] - ref[q]) / nr
        assert err <= rtol, "param %d: relative error %.3g" % (q, err)
        assert np.max(np.abs(g[q] - ref[q])) <= elem * np.max(np.abs(ref[q])), q


def oracle_loss_grad(sc, theta, Y, K, stride):
    P, V = oracle.forward(sc["lane_off"], sc["length"], theta, sc["p_init"], sc["v_init"], K, DT, A_MIN)
    L, gP = oracle.mse_seed(P, Y, stride)
    g, gp, gv = oracle.adjoint(sc["lane_off"], sc["length"], theta, K, DT, P, V, gP, None, A_MIN)
    return L, g, gp, gv, P


def noisy_targets(sc, K, stride, rng):
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    n_obs = K // stride
    N = P.shape[1]
    return synth.f32(P[stride::stride][:n_obs] + rng.normal(0, 0.5, size=(n_obs, N)))


def run_loss_grad(api, sc, theta, Y, K, stride, ctx=None):
    scn = scene_of(api, sc)
    loss, g, gp, gv = api.loss_grad(cuda(theta), cuda(sc["p_init"]), cuda(sc["v_init"]), scn, K, DT,
                                    cuda(Y) if Y.size else None, stride, A_MIN, ctx=ctx)
    torch.cuda.synchronize()
    return loss.item(), g.double().cpu().numpy(), gp.double().cpu().numpy(), gv.double().cpu().numpy()


# ---------------------------------------------------------------------------
# config 0: 10 lanes x 100 vehicles, 100 steps
# ---------------------------------------------------------------------------

def test_forward_config0(api):
    sc = synth.config0()
    K = sc["K"]
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    traj, vtraj = api.simulate(cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc),
                               K, DT, A_MIN, want_speed=True)
    traj = traj.double().cpu().numpy()
    vtraj = vtraj.double().cpu().numpy()
    assert np.max(np.abs(traj - P)) <= POS_TOL
    assert np.max(np.abs(vtraj - V)) <= 1e-4
    np.testing.assert_array_equal(traj[0], sc["p_init"])


@pytest.mark.parametrize("init", ["plain", "near_truth"])
def test_loss_grad_config0(api, init):
    sc = synth.config0()
    K, s = sc["K"], sc["obs_stride"]
    Y = noisy_targets(sc, K, s, np.random.default_rng(100))
    if init == "plain":
        theta = synth.plain_init(1000)
    else:
        theta = synth.f32(sc["theta_true"] * np.random.default_rng(101).uniform(0.95, 1.05, size=(6, 1000)))
        theta[5] = 4.0
    L, g, gp, gv, _ = oracle_loss_grad(sc, theta, Y, K, s)
    Lg, gg, gpg, gvg = run_loss_grad(api, sc, theta, Y, K, s)
    assert Lg == pytest.approx(L, rel=1e-5)
    grad_close(gg, g)
    grad_close(np.stack([gpg, gvg]), np.stack([gp, gv]), rows=range(2))


@pytest.mark.parametrize("ckpt", [8, 23])
def test_backward_dense_seeds(api, ckpt):
    # ckpt 23 exceeds the shared-memory tape depth: tape blocks restarted
    # from sub-checkpoints
    sc = synth.config0()
    K = 60
    rng = np.random.default_rng(102)
    N = 1000
    gP = synth.f32(rng.normal(size=(K + 1, N)))
    gV = synth.f32(rng.normal(size=(K + 1, N)))
    theta = sc["theta_true"]
    P, V = oracle.forward(sc["lane_off"], sc["length"], theta, sc["p_init"], sc["v_init"], K, DT, A_MIN)
    g, gp, gv = oracle.adjoint(sc["lane_off"], sc["length"], theta, K, DT, P, V, gP, gV, A_MIN)
    gg, gpg, gvg = api.backward(cuda(theta), cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K, DT,
                                cuda(gP), cuda(gV), A_MIN, ctx=api.Context(ckpt_interval=ckpt))
    grad_close(gg.double().cpu().numpy(), g)
    grad_close(np.stack([gpg.double().cpu().numpy(), gvg.double().cpu().numpy()]), np.stack([gp, gv]),
               rows=range(2))


def test_autograd_function(api):
    sc = synth.config0()
    K = 40
    rng = np.random.default_rng(103)
    w = synth.f32(rng.normal(size=(K + 1, 1000)))
    th = cuda(sc["theta_true"]).requires_grad_(True)
    p0 = cuda(sc["p_init"]).requires_grad_(True)
    v0 = cuda(sc["v_init"]).requires_grad_(True)
    traj = api.IdmFunction.apply(th, p0, v0, scene_of(api, sc), K, DT, A_MIN)
    (traj * cuda(w)).sum().backward()
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    g, gp, gv = oracle.adjoint(sc["lane_off"], sc["length"], sc["theta_true"], K, DT, P, V, w, None, A_MIN)
    grad_close(th.grad.double().cpu().numpy(), g)
    grad_close(np.stack([p0.grad.double().cpu().numpy(), v0.grad.double().cpu().numpy()]), np.stack([gp, gv]),
               rows=range(2))


# ---------------------------------------------------------------------------
# edge shapes, kernel variants, checkpoint intervals
# ---------------------------------------------------------------------------

EDGE_COUNTS = [1, 2, 3, 33, 0, 17, 31, 32, 1, 5]


@pytest.mark.parametrize("vpt,G,C", [(2, 1, 1), (2, 2, 7), (4, 4, 16), (2, 4, 5), (0, 0, 64), (4, 1, 8), (8, 2, 3)])
def test_edge_lanes(api, vpt, G, C):
    rng = np.random.default_rng(104)
    sc = synth.make_scene(EDGE_COUNTS, rng)
    K, s = 37, 3
    Y = noisy_targets(sc, K, s, rng)
    N = int(sc["lane_off"][-1])
    theta = synth.f32(sc["theta_true"] * rng.uniform(0.8, 1.2, size=(6, N)))
    L, g, gp, gv, _ = oracle_loss_grad(sc, theta, Y, K, s)
    ctx = api.Context(vpt=vpt, warps_per_segment=G, ckpt_interval=C, warps_per_block=8)
    Lg, gg, gpg, gvg = run_loss_grad(api, sc, theta, Y, K, s, ctx=ctx)
    assert ctx.check_status() == 0
    assert Lg == pytest.approx(L, rel=1e-5)
    grad_close(gg, g)
    grad_close(np.stack([gpg, gvg]), np.stack([gp, gv]), rows=range(2))


@pytest.mark.parametrize("counts,vpt,G", [([1000, 37, 500], 4, 8), ([2048, 3], 8, 8), ([300, 200, 129], 2, 8)])
def test_long_lanes_multiwarp(api, counts, vpt, G):
    """Lanes longer than one warp's slots: leader values and follower terms
    cross warp boundaries inside a segment every step."""
    rng = np.random.default_rng(115)
    sc = synth.make_scene(counts, rng)
    K, s = 24, 2
    Y = noisy_targets(sc, K, s, rng)
    N = int(sc["lane_off"][-1])
    theta = synth.f32(sc["theta_true"] * rng.uniform(0.9, 1.1, size=(6, N)))
    L, g, gp, gv, P = oracle_loss_grad(sc, theta, Y, K, s)
    ctx = api.Context(vpt=vpt, warps_per_segment=G, ckpt_interval=5, warps_per_block=8)
    Lg, gg, gpg, gvg = run_loss_grad(api, sc, theta, Y, K, s, ctx=ctx)
    assert ctx.check_status() == 0
    assert Lg == pytest.approx(L, rel=1e-5)
    grad_close(gg, g)
    grad_close(np.stack([gpg, gvg]), np.stack([gp, gv]), rows=range(2))
    traj = api.simulate(cuda(theta), cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K, DT, A_MIN,
                        ctx=ctx).double().cpu().numpy()
    # positions reach tens of km behind a 1,000-vehicle lane head, where one
    # float32 ulp of the output exceeds 1e-3 m: allow 1e-3 m plus 2 ulp
    np.testing.assert_allclose(traj, P, rtol=2.4e-7, atol=POS_TOL)


def test_single_step(api):
    rng = np.random.default_rng(105)
    sc = synth.make_scene([4, 9], rng)
    Y = noisy_targets(sc, 1, 1, rng)
    L, g, gp, gv, _ = oracle_loss_grad(sc, sc["theta_true"], Y, 1, 1)
    Lg, gg, gpg, gvg = run_loss_grad(api, sc, sc["theta_true"], Y, 1, 1)
    assert Lg == pytest.approx(L, rel=1e-5)
    grad_close(np.stack([gpg, gvg]), np.stack([gp, gv]), rows=range(2))
    grad_close(gg, g, rows=[0, 3, 5])


def test_stride_beyond_horizon(api):
    rng = np.random.default_rng(106)
    sc = synth.make_scene([6, 6], rng)
    Lg, gg, gpg, gvg = run_loss_grad(api, sc, sc["theta_true"], np.zeros((0, 12)), 9, 10)
    assert Lg == 0.0 and np.all(gg == 0.0) and np.all(gpg == 0.0) and np.all(gvg == 0.0)


def test_long_horizon_positions(api):
    """1,000 steps: the float32 pair keeps positions close to FP64."""
    rng = np.random.default_rng(107)
    sc = synth.make_scene([100] * 4, rng)
    K = 1000
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    traj = api.simulate(cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K, DT,
                        A_MIN).double().cpu().numpy()
    assert np.max(np.abs(traj - P)) <= 5e-3


def test_long_horizon_fit_then_predict(api):
    """Fit on the first 400 of 600 steps with checkpoints every 20 steps
    (about sqrt(400)), then predict all 600 steps with the fitted
    parameters: the fit matches the oracle's fit, the prediction the
    oracle's simulation of the same parameters."""
    rng = np.random.default_rng(112)
    sc = synth.make_scene([50] * 8, rng)
    N = 400
    K_fit, K_all = 400, 600
    P_true, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K_all, DT,
                               A_MIN)
    Y = synth.f32(P_true[1:K_fit + 1] + rng.normal(0, 0.5, size=(K_fit, N)))
    th0 = synth.plain_init(N)
    n_iter = 6
    th_ref, _ = oracle.fit(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K_fit, DT, Y, 1, n_iter,
                           0.1, 0.01, synth.BOX_LO, synth.BOX_HI, A_MIN)
    ctx = api.Context(ckpt_interval=20)
    th = cuda(th0)
    api.fit(th, cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K_fit, DT, cuda(Y), 1, n_iter, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.check_status() == 0
    th_gpu = th.double().cpu().numpy()
    np.testing.assert_allclose(th_gpu, th_ref, rtol=1e-4, atol=1e-5)
    traj = api.simulate(th, cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K_all, DT, A_MIN, ctx=ctx)
    P_pred, _ = oracle.forward(sc["lane_off"], sc["length"], th_gpu, sc["p_init"], sc["v_init"], K_all, DT, A_MIN)
    assert np.max(np.abs(traj.double().cpu().numpy() - P_pred)) <= 5e-3


# ---------------------------------------------------------------------------
# fit, layout
# ---------------------------------------------------------------------------

def test_fit_config0(api):
    sc = synth.config0()
    K, s = sc["K"], sc["obs_stride"]
    Y = noisy_targets(sc, K, s, np.random.default_rng(108))
    n_iter = 5
    th0 = synth.plain_init(1000)
    th_ref, hist_ref = oracle.fit(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K, DT, Y, s, n_iter,
                                  0.1, 0.01, synth.BOX_LO, synth.BOX_HI, A_MIN)
    th = cuda(th0)
    hist = api.fit(th, cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K, DT, cuda(Y), s, n_iter, 0.1,
                   0.01, synth.BOX_LO, synth.BOX_HI, A_MIN)
    torch.cuda.synchronize()
    np.testing.assert_allclose(hist.cpu().numpy(), hist_ref, rtol=1e-5)
    np.testing.assert_allclose(th.double().cpu().numpy(), th_ref, rtol=1e-4, atol=1e-5)


def test_fit_eval_history(api):
    # idm_fit_eval: same updates as idm_fit; the eval history is the loss of
    # each iterate against the second target set (here the clean truth,
    # checked against the oracle at the iterates the oracle fit produces).
    sc = synth.config0()
    K, s = sc["K"], 2
    P_true, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT,
                               A_MIN)
    clean = synth.f32(P_true[s::s][: K // s])
    Y = noisy_targets(sc, K, s, np.random.default_rng(111))
    n_iter = 4
    th0 = synth.plain_init(1000)
    ref_eval = []
    for m in range(n_iter):  # iterate m of the n_iter schedule: replay the first m updates in the oracle
        th_m = th0 if m == 0 else _oracle_fit_prefix(sc, th0, Y, K, s, n_iter, m)
        Pm, _ = oracle.forward(sc["lane_off"], sc["length"], th_m, sc["p_init"], sc["v_init"], K, DT, A_MIN)
        ref_eval.append(oracle.mse_seed(Pm, clean, s)[0])
    th_a, th_b = cuda(th0), cuda(th0)
    hist_a = api.fit(th_a, cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K, DT, cuda(Y), s, n_iter)
    hist_b, ev = api.fit(th_b, cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K, DT, cuda(Y), s, n_iter,
                         eval_targets=cuda(clean))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hist_a.cpu().numpy(), hist_b.cpu().numpy())
    np.testing.assert_array_equal(th_a.cpu().numpy(), th_b.cpu().numpy())
    np.testing.assert_allclose(ev.cpu().numpy(), np.array(ref_eval), rtol=1e-4)
    # with the fitting targets as the second set, both histories agree
    th_c = cuda(th0)
    hist_c, ev_c = api.fit(th_c, cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), K, DT, cuda(Y), s,
                           n_iter, eval_targets=cuda(Y))
    np.testing.assert_allclose(ev_c.cpu().numpy(), hist_c.cpu().numpy(), rtol=1e-5)


def _oracle_fit_prefix(sc, th0, Y, K, s, n_iter, m):
    """Parameters after the first m Adam updates of an n_iter-iteration fit
    (oracle steps with the n_iter learning-rate schedule)."""
    th = np.array(th0, dtype=np.float64, copy=True)
    N = th.shape[1]
    m1, v1 = np.zeros((5, N)), np.zeros((5, N))
    for it in range(m):
        P, V = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, DT, A_MIN)
        _, gP = oracle.mse_seed(P, Y, s)
        g, _, _ = oracle.adjoint(sc["lane_off"], sc["length"], th, K, DT, P, V, gP, None, A_MIN)
        th5 = np.ascontiguousarray(th[:5])
        oracle.adam_step(th5, np.ascontiguousarray(g[:5]), m1, v1, it + 1, oracle.lr_schedule(it, n_iter, 0.1, 0.01),
                         synth.BOX_LO, synth.BOX_HI)
        th[:5] = th5
    return th


@pytest.mark.parametrize("N,R", [(1, 7), (5, 3), (2047, 2), (4099, 5), (100003, 3)])
def test_gather_rows_bitexact(api, N, R):
    """idm_gather_rows: dst[r][j] = src[r][perm[j]] over row-major [R][N]
    arrays, bit for bit, for sizes that end mid-chunk and rows shorter than a
    chunk."""
    from paper_2412_16750_gb300 import lib
    rng = np.random.default_rng(N + R)
    perm = rng.permutation(N).astype(np.int32)
    src = rng.normal(size=(R, N)).astype(np.float32)
    ctx = api.Context()
    d = torch.full((R, N), float("nan"), device="cuda")
    lib.idm_gather_rows(ctx.handle, N, R, cuda(perm, torch.int32), cuda(src), d, torch.cuda.current_stream())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), src[:, perm])


def test_layout_bitexact(api):
    rng = np.random.default_rng(109)
    N, L = 20000, 613
    lane = rng.integers(0, L, size=N).astype(np.int32)
    pos = synth.f32(rng.uniform(-3000, 0, size=N))
    pos[::11] = pos[3]
    pos[::13] = 0.0
    pos[::17] = -0.0
    perm_ref, off_ref = oracle.layout(lane, pos, L)
    perm, off, mx = api.layout(cuda(lane, torch.int32), cuda(pos), L)
    np.testing.assert_array_equal(perm.cpu().numpy(), perm_ref)
    np.testing.assert_array_equal(off.cpu().numpy(), off_ref)
    assert int(mx.item()) == int(np.diff(off_ref).max())
    dst = api.gather(perm, [cuda(pos)])[0].cpu().numpy()
    np.testing.assert_array_equal(dst, pos[perm_ref].astype(np.float32))


# ---------------------------------------------------------------------------
# errors and status
# ---------------------------------------------------------------------------

def test_argument_errors(api):
    from paper_2412_16750_gb300 import lib
    sc = synth.make_scene([3, 3], np.random.default_rng(110))
    scn = scene_of(api, sc)
    th, p0, v0 = cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"])
    with pytest.raises(lib.IdmError) as e:
        api.simulate(th, p0, v0, scn, 0, DT)
    assert e.value.code == lib.IDM_ERR_ARG
    with pytest.raises(lib.IdmError) as e:
        api.simulate(th, p0, v0, scn, 5, -0.1)
    assert e.value.code == lib.IDM_ERR_ARG
    with pytest.raises(lib.IdmError) as e:
        api.loss_grad(th, p0, v0, scn, 5, DT, cuda(np.zeros((5, 6))), 0)
    assert e.value.code == lib.IDM_ERR_ARG
    big = api.Scene(scn.lane_off, scn.length, 3000)
    with pytest.raises(lib.IdmError) as e:
        api.simulate(th, p0, v0, big, 5, DT)
    assert e.value.code == lib.IDM_ERR_ARG
    ctx = api.Context(workspace_cap_bytes=64)
    with pytest.raises(lib.IdmError) as e:
        api.loss_grad(th, p0, v0, scn, 5, DT, cuda(np.zeros((5, 6))), 1, ctx=ctx)
    assert e.value.code == lib.IDM_ERR_WORKSPACE


def test_device_status_lane_too_long(api):
    from paper_2412_16750_gb300 import lib
    sc = synth.make_scene([70, 3], np.random.default_rng(111))
    ctx = api.Context(vpt=2, warps_per_segment=1)
    scn = api.Scene(cuda(sc["lane_off"], torch.int32), cuda(sc["length"]), 32)  # understated max_lane
    traj = api.simulate(cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"]), scn, 5, DT, ctx=ctx)
    rc, flags = ctx.status()
    assert rc == lib.IDM_ERR_LANE and flags & lib.IDM_STATUS_LANE_TOO_LONG
    # the short lane is still simulated
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], 5, DT, A_MIN)
    np.testing.assert_allclose(traj[:, 70:].double().cpu().numpy(), P[:, 70:], atol=POS_TOL)
    assert ctx.status()[0] == lib.IDM_OK  # cleared


def test_device_status_bad_lane_off(api):
    from paper_2412_16750_gb300 import lib
    sc = synth.make_scene([4, 4, 4], np.random.default_rng(112))
    ctx = api.Context()
    bad = np.array([0, 9, 4, 12], dtype=np.int32)  # not monotone
    scn = api.Scene(cuda(bad, torch.int32), cuda(sc["length"]), 9)
    api.simulate(cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"]), scn, 3, DT, ctx=ctx)
    rc, flags = ctx.status()
    assert rc == lib.IDM_ERR_LANE and flags & lib.IDM_STATUS_BAD_LANE_OFF
    over = np.array([0, 4, 8, 99], dtype=np.int32)  # past the last vehicle: never read
    scn = api.Scene(cuda(over, torch.int32), cuda(sc["length"]), 91)
    api.simulate(cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"]), scn, 3, DT, ctx=ctx)
    rc, flags = ctx.status()
    assert rc == lib.IDM_ERR_LANE and flags & lib.IDM_STATUS_BAD_LANE_OFF


def test_device_status_nonfinite(api):
    from paper_2412_16750_gb300 import lib
    sc = synth.make_scene([5], np.random.default_rng(113))
    th = sc["theta_true"].copy()
    th[3, 2] = np.nan
    ctx = api.Context()
    api.simulate(cuda(th), cuda(sc["p_init"]), cuda(sc["v_init"]), scene_of(api, sc), 4, DT, ctx=ctx)
    rc, flags = ctx.status()
    assert rc == lib.IDM_ERR_NONFINITE and flags & lib.IDM_STATUS_NONFINITE


# ---------------------------------------------------------------------------
# full size: 20,000 lanes x 100 vehicles x 1,000 steps, sampled lanes
# ---------------------------------------------------------------------------

def test_full_size_sampled_lanes(api):
    """The paper-scale workload in the launch configuration the benchmark
    uses; the oracle recomputes 12 sampled lanes (lanes are independent)."""
    sc = synth.config1()
    K = sc["K"]
    N = int(sc["lane_off"][-1])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(20241217)
    p0, v0 = cuda(sc["p_init"]), cuda(sc["v_init"])
    k = torch.arange(1, K + 1, device="cuda", dtype=torch.float32)[:, None]
    Y = (p0[None, :] + k * DT * v0[None, :] + 0.5 * torch.randn((K, N), device="cuda", generator=gen)).contiguous()
    theta = synth.plain_init(N)
    th = cuda(theta)
    loss, g, gp, gv = api.loss_grad(th, p0, v0, scene_of(api, sc), K, DT, Y, 1, A_MIN)
    torch.cuda.synchronize()
    lanes = np.random.default_rng(114).choice(20000, size=12, replace=False)
    lo = sc["lane_off"]
    g = g.double().cpu().numpy()
    gp = gp.double().cpu().numpy()
    for l in lanes:
        a, e = int(lo[l]), int(lo[l + 1])
        sub = dict(lane_off=np.array([0, e - a], dtype=np.int32), length=sc["length"][a:e], p_init=sc["p_init"][a:e],
                   v_init=sc["v_init"][a:e])
        Ys = Y[:, a:e].double().cpu().numpy()
        L, gr, gpr, gvr, P = oracle_loss_grad(sub, theta[:, a:e], Ys, K, 1)
        grad_close(g[:, a:e], gr)
        grad_close(gp[None, a:e], gpr[None], rows=[0])
    # forward positions of the sampled lanes over all 1,000 steps
    traj = api.simulate(th, p0, v0, scene_of(api, sc), K, DT, A_MIN)
    for l in lanes[:4]:
        a, e = int(lo[l]), int(lo[l + 1])
        P, _ = oracle.forward(np.array([0, e - a], dtype=np.int32), sc["length"][a:e], theta[:, a:e],
                              sc["p_init"][a:e], sc["v_init"][a:e], K, DT, A_MIN)
        assert np.max(np.abs(traj[:, a:e].double().cpu().numpy() - P)) <= 5e-3


def braking_scene(seed, n_lanes=30):
    """Lanes of three: a stopped leader, a follower creeping (v < 1 m/s, so
    the -v/dt bound is active) a few centimetres behind it, a third vehicle
    behind that.  The follower's next speed rounds to a few ulps below 0."""
    rng = np.random.default_rng(seed)
    p, v, L = [], [], []
    for _ in range(n_lanes):
        g1, g2 = rng.uniform(0.02, 0.5), rng.uniform(0.5, 3.0)
        p += [0.0, -(5.0 + g1), -(10.0 + g1 + g2)]
        v += [0.0, rng.uniform(0.05, 0.9), rng.uniform(0.0, 0.9)]
        L += [5.0, 5.0, 5.0]
    N = 3 * n_lanes
    th = np.vstack([rng.uniform(lo, hi, N) for lo, hi in synth.TRUE_RANGES] + [np.full(N, 4.0)])
    return dict(lane_off=synth.lane_offsets([3] * n_lanes), length=synth.f32(L), p_init=synth.f32(p),
                v_init=synth.f32(v), theta_true=synth.f32(th))


def test_braking_to_rest_delta_gradient(api):
    sc = braking_scene(71)
    K, s = 30, 1
    Y = noisy_targets(sc, K, s, np.random.default_rng(72))
    th = synth.plain_init(len(sc["length"]))
    L, g_ref, gp_ref, gv_ref, _ = oracle_loss_grad(sc, th, Y, K, s)
    loss, g, gp, gv = run_loss_grad(api, sc, th, Y, K, s)
    assert np.isfinite(g).all() and np.isfinite(gp).all() and np.isfinite(gv).all()
    assert abs(loss - L) <= 1e-5 * L
    grad_close(g, g_ref)
    assert api.default_context().check_status() == 0


# ---------------------------------------------------------------------------
# config 4's fit window: 2,000 steps, checkpoints every 45 steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("init", ["near_truth", "plain"])
def test_long_horizon_gradients_2000_steps(api, init):
    """Loss and gradients over 2,000 steps, every step observed, with the
    checkpoint interval of the long-horizon fit (45 steps: tape blocks
    restarted from sub-checkpoints), element by element against the FP64
    adjoint.  The per-vehicle gradient sums run over 2,000 terms; their
    compensated accumulation keeps them at the 1e-4 bar."""
    rng = np.random.default_rng(116)
    counts = [100, 100, 37, 100, 64, 100, 1, 100, 100, 3, 100, 100]   # ragged lanes, several segments
    sc = synth.make_scene(counts, rng)
    N, K = int(sum(counts)), 2000
    Y = noisy_targets(sc, K, 1, rng)
    if init == "plain":
        theta = synth.plain_init(N)
    else:
        theta = synth.f32(sc["theta_true"] * rng.uniform(0.97, 1.03, size=(6, N)))
        theta[5] = 4.0
    L, g, gp, gv, _ = oracle_loss_grad(sc, theta, Y, K, 1)
    ctx = api.Context(ckpt_interval=45)
    Lg, gg, gpg, gvg = run_loss_grad(api, sc, theta, Y, K, 1, ctx=ctx)
    assert ctx.check_status() == 0
    assert Lg == pytest.approx(L, rel=1e-5)
    grad_close(gg, g)
    grad_close(np.stack([gpg, gvg]), np.stack([gp, gv]), rows=range(2))


# ---------------------------------------------------------------------------
# event counters: gap-floor hits and the kink band of the lower bound
# ---------------------------------------------------------------------------

def event_scene():
    """Lanes built to hit the gap floor and to sit near v = 1 m/s (the kink of
    max(-v/dt, a_min) at dt = 0.1 s, a_min = -10):
      * lone vehicles with v0 = 0.98, 1.0, 1.03 m/s starting at their v0:
        every step in the band;
      * a follower 3 cm behind a faster leader (floor at its first steps),
        braking hard through the band;
      * a queue starting from rest (accelerating through 1 m/s), its followers
        5-8 cm apart."""
    p, v, th = [], [], []
    counts = []
    base = [30.0, 1.5, 2.0, 1.0, 2.0, 4.0]
    for v0 in (0.98, 1.0, 1.03):
        p.append(0.0); v.append(v0); th.append([v0] + base[1:]); counts.append(1)
    p += [0.0, -5.03]; v += [10.0, 9.5]; th += [base, base]; counts.append(2)
    q = [0.0]
    for gap in (0.05, 0.07, 0.06, 0.08):
        q.append(q[-1] - 5.0 - gap)
    p += q; v += [0.0] * len(q); th += [base] * len(q); counts.append(len(q))
    N = len(p)
    return dict(lane_off=synth.lane_offsets(counts), length=synth.f32(np.full(N, 5.0)), p_init=synth.f32(p),
                v_init=synth.f32(v), theta_true=synth.f32(np.array(th).T))


def oracle_event_bounds(sc, K, margin_gap=1e-4, margin_kink=1e-3):
    """Counts over steps 0..K-1 from the oracle's trajectory (gap of a
    follower = P_leader - P - length_leader; the kink quantity -v/dt - a_min),
    as [definitely inside, possibly inside] given the FP32/FP64 difference of
    the states (well below the margins)."""
    P, V = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    N = P.shape[1]
    lo = sc["lane_off"]
    head = np.zeros(N, dtype=bool)
    head[[int(lo[l]) for l in range(len(lo) - 1) if lo[l + 1] > lo[l]]] = True
    gap = np.full((K, N), np.inf)
    gap[:, 1:] = P[:K, :-1] - P[:K, 1:] - sc["length"][None, :-1]
    gap[:, head] = np.inf
    x = np.abs(-V[:K] / DT - A_MIN)
    floor = (int((gap < 0.1 - margin_gap).sum()), int((gap < 0.1 + margin_gap).sum()))
    kink = (int((x < 0.5 - margin_kink).sum()), int((x < 0.5 + margin_kink).sum()))
    return floor, kink


def test_event_counts_against_oracle(api):
    sc = event_scene()
    K = 200
    (f_lo, f_hi), (k_lo, k_hi) = oracle_event_bounds(sc, K)
    assert f_lo > 0 and k_lo >= 3 * K    # the scene does exercise both counters
    ctx = api.Context()
    th, p0, v0 = cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"])
    api.simulate(th, p0, v0, scene_of(api, sc), K, DT, A_MIN, ctx=ctx)
    assert ctx.event_counts() == {"gap_floor_hits": 0, "kink_near": 0}      # off by default
    ctx.set_event_counting(True)
    api.simulate(th, p0, v0, scene_of(api, sc), K, DT, A_MIN, ctx=ctx)
    got = ctx.event_counts()
    assert f_lo <= got["gap_floor_hits"] <= f_hi, (got, f_lo, f_hi)
    assert k_lo <= got["kink_near"] <= k_hi, (got, k_lo, k_hi)
    assert ctx.event_counts() == {"gap_floor_hits": 0, "kink_near": 0}      # read clears
    for _ in range(2):                                                      # counts accumulate until read
        api.simulate(th, p0, v0, scene_of(api, sc), K, DT, A_MIN, ctx=ctx)
    assert ctx.event_counts() == {"gap_floor_hits": 2 * got["gap_floor_hits"], "kink_near": 2 * got["kink_near"]}
    # the batched forward counts the same events (two copies of the scene as scenarios)
    lanes = np.diff(sc["lane_off"])
    L = len(lanes)
    b = api.Batch(np.array([0, L, 2 * L], np.int32), np.array([K, K], np.int32), np.array([DT, DT], np.float32),
                  np.array([1, 1], np.int32), synth.lane_offsets(np.concatenate([lanes, lanes])),
                  np.concatenate([sc["length"], sc["length"]]), A_MIN)
    two = lambda x: cuda(np.concatenate([x, x], axis=-1))
    api.batch_forward(two(sc["theta_true"]), two(sc["p_init"]), two(sc["v_init"]), b, ctx=ctx)
    assert ctx.event_counts() == {"gap_floor_hits": 2 * got["gap_floor_hits"], "kink_near": 2 * got["kink_near"]}
    assert ctx.check_status() == 0
