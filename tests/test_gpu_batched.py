"""GPU parity of the batched uneven-scenario entry points against the FP64
oracle run scenario by scenario (scenarios are independent)."""
import numpy as np
import pytest

import oracle
from paper_2412_16750_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = float(np.float32(0.1))
A_MIN = -10.0


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16750_gb300 import api as _api
    return _api


def cuda(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def sub_scene(sc, s):
    lo = sc["lane_off"]
    l0, l1 = sc["scen_lane_off"][s], sc["scen_lane_off"][s + 1]
    a, e = lo[l0], lo[l1]
    return dict(lane_off=(lo[l0:l1 + 1] - a).astype(np.int32), length=sc["length"][a:e], p_init=sc["p_init"][a:e],
                v_init=sc["v_init"][a:e]), a, e


def small_batch(seed, n_scen=14):
    rng = np.random.default_rng(seed)
    lanes = rng.integers(1, 5, size=n_scen)
    counts = [rng.integers(1, 45, size=int(L)) for L in lanes]
    K = rng.integers(3, 41, size=n_scen)
    stride = rng.integers(1, 5, size=n_scen)
    stride[0] = 50  # no observation in the first scenario
    return synth.make_batch(lanes, counts, K, stride, rng), rng


def targets_for(sc, rng):
    """Per-scenario targets (truth + noise) from the oracle, concatenated."""
    blocks = []
    for s in range(len(sc["K"])):
        sub, a, e = sub_scene(sc, s)
        K, st = int(sc["K"][s]), int(sc["obs_stride"][s])
        P, _ = oracle.forward(sub["lane_off"], sub["length"], sc["theta_true"][:, a:e], sub["p_init"], sub["v_init"],
                              K, DT, A_MIN)
        n_obs = K // st
        blocks.append(synth.f32(P[st::st][:n_obs] + rng.normal(0, 0.5, size=(n_obs, e - a))).ravel())
    return np.concatenate(blocks)


def batch_of(api, sc):
    return api.Batch(sc["scen_lane_off"], sc["K"], sc["dt"], sc["obs_stride"], sc["lane_off"], sc["length"], A_MIN)


@pytest.mark.parametrize("shape", [(0, 0, 4), (2, 1, 4), (4, 4, 4), (4, 4, 30)])
def test_batch_loss_grad_parity(api, shape):
    # the last shape's checkpoint interval exceeds the tape depth (tape blocks)
    sc, rng = small_batch(200)
    Y = targets_for(sc, rng)
    N = int(sc["lane_off"][-1])
    theta = synth.f32(sc["theta_true"] * rng.uniform(0.85, 1.15, size=(6, N)))
    ctx = api.Context(vpt=shape[0], warps_per_segment=shape[1], ckpt_interval=shape[2])
    b = batch_of(api, sc)
    sl, tot, g, gp, gv = api.batch_loss_grad(cuda(theta), cuda(sc["p_init"]), cuda(sc["v_init"]), b, cuda(Y), ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.check_status() == 0
    sl = sl.cpu().numpy()
    g = g.double().cpu().numpy()
    gp = gp.double().cpu().numpy()
    off = 0
    total = 0.0
    for s in range(len(sc["K"])):
        sub, a, e = sub_scene(sc, s)
        K, st = int(sc["K"][s]), int(sc["obs_stride"][s])
        n_obs = K // st
        Ys = Y[off:off + n_obs * (e - a)].reshape(n_obs, e - a) if n_obs else np.zeros((0, e - a))
        off += n_obs * (e - a)
        P, V = oracle.forward(sub["lane_off"], sub["length"], theta[:, a:e], sub["p_init"], sub["v_init"], K, DT, A_MIN)
        L, gP = oracle.mse_seed(P, Ys, st)
        gr, gpr, gvr = oracle.adjoint(sub["lane_off"], sub["length"], theta[:, a:e], K, DT, P, V, gP, None, A_MIN)
        total += L
        assert sl[s] == pytest.approx(L, rel=1e-5, abs=1e-12)
        scale = max(np.abs(gr).max(), 1e-30)
        np.testing.assert_allclose(g[:, a:e], gr, rtol=0, atol=2e-4 * scale)
        np.testing.assert_allclose(gp[a:e], gpr, rtol=0, atol=2e-4 * max(np.abs(gpr).max(), 1e-30))
    assert tot.item() == pytest.approx(total, rel=1e-5)


def test_batch_forward_parity(api):
    sc, rng = small_batch(201)
    N = int(sc["lane_off"][-1])
    b = batch_of(api, sc)
    traj = api.batch_forward(cuda(sc["theta_true"]), cuda(sc["p_init"]), cuda(sc["v_init"]), b).double().cpu().numpy()
    for s in range(len(sc["K"])):
        sub, a, e = sub_scene(sc, s)
        K = int(sc["K"][s])
        P, _ = oracle.forward(sub["lane_off"], sub["length"], sc["theta_true"][:, a:e], sub["p_init"], sub["v_init"],
                              K, DT, A_MIN)
        blk = traj[b.traj_off[s]:b.traj_off[s + 1]].reshape(K + 1, e - a)
        assert np.max(np.abs(blk - P)) <= 1e-3


def test_batch_fit_parity(api):
    sc, rng = small_batch(202, n_scen=6)
    Y = targets_for(sc, rng)
    N = int(sc["lane_off"][-1])
    th0 = synth.plain_init(N)
    th = cuda(th0)
    b = batch_of(api, sc)
    hist, sl = api.batch_fit(th, cuda(sc["p_init"]), cuda(sc["v_init"]), b, cuda(Y), 4)
    torch.cuda.synchronize()
    th = th.double().cpu().numpy()
    hist = hist.cpu().numpy()
    # the summed loss is the sum of independent per-scenario fits (Adam is per vehicle)
    off = 0
    ref_hist = np.zeros(4)
    for s in range(len(sc["K"])):
        sub, a, e = sub_scene(sc, s)
        K, st = int(sc["K"][s]), int(sc["obs_stride"][s])
        n_obs = K // st
        Ys = Y[off:off + n_obs * (e - a)].reshape(max(n_obs, 1) if n_obs else 1, e - a) if n_obs else np.zeros((1, e - a))
        off += n_obs * (e - a)
        thr, hr = oracle.fit(sub["lane_off"], sub["length"], th0[:, a:e], sub["p_init"], sub["v_init"], K, DT, Ys, st,
                             4, 0.1, 0.01, synth.BOX_LO, synth.BOX_HI, A_MIN)
        ref_hist += hr
        np.testing.assert_allclose(th[:, a:e], thr, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(hist, ref_hist, rtol=1e-5)


def test_config2_full_size_sampled(api):
    """4,096 uneven scenarios in one launch; 8 sampled scenarios recomputed by
    the oracle.  Targets: constant-velocity kinematics + noise, drawn on the
    device with a seeded generator and copied for the oracle."""
    sc = synth.config2()
    b = batch_of(api, sc)
    N = b.n_vehicles
    gen = torch.Generator(device="cuda")
    gen.manual_seed(20241218)
    tgt = torch.empty(int(b.tgt_off[-1]), device="cuda", dtype=torch.float32)
    p0, v0 = cuda(sc["p_init"]), cuda(sc["v_init"])
    for s in range(b.n_scen):
        a, e = int(b.veh_off[s]), int(b.veh_off[s + 1])
        st, n_obs = int(b.obs_stride[s]), int(b.n_obs[s])
        k = (torch.arange(1, n_obs + 1, device="cuda", dtype=torch.float32) * st)[:, None]
        blk = p0[None, a:e] + k * DT * v0[None, a:e] + 0.5 * torch.randn((n_obs, e - a), device="cuda", generator=gen)
        tgt[b.tgt_off[s]:b.tgt_off[s + 1]] = blk.reshape(-1)
    theta = synth.plain_init(N)
    sl, tot, g, gp, gv = api.batch_loss_grad(cuda(theta), p0, v0, b, tgt)
    torch.cuda.synchronize()
    g = g.double().cpu().numpy()
    sl = sl.cpu().numpy()
    for s in np.random.default_rng(203).choice(b.n_scen, size=8, replace=False):
        sub, a, e = sub_scene(sc, s)
        K, st = int(sc["K"][s]), int(sc["obs_stride"][s])
        n_obs = K // st
        Ys = tgt[b.tgt_off[s]:b.tgt_off[s + 1]].double().cpu().numpy().reshape(n_obs, e - a)
        P, V = oracle.forward(sub["lane_off"], sub["length"], theta[:, a:e], sub["p_init"], sub["v_init"], K, DT, A_MIN)
        L, gP = oracle.mse_seed(P, Ys, st)
        gr, _, _ = oracle.adjoint(sub["lane_off"], sub["length"], theta[:, a:e], K, DT, P, V, gP, None, A_MIN)
        assert sl[s] == pytest.approx(L, rel=1e-5)
        for q in range(6):
            nr = np.linalg.norm(gr[q])
            if nr > 0:
                assert np.linalg.norm(g[q, a:e] - gr[q]) / nr <= 1e-4


def test_autotuned_shape_keeps_parity(api, tmp_path):
    """The autotuner times the batched loss + gradient over candidate shapes,
    caches the fastest and applies it; results under that shape still match
    the oracle, and a second call is served from the cache."""
    from paper_2412_16750_gb300 import tune
    sc, rng = small_batch(203)
    Y = cuda(targets_for(sc, rng))
    N = int(sc["lane_off"][-1])
    theta = cuda(synth.f32(sc["theta_true"] * rng.uniform(0.9, 1.1, size=(6, N))))
    p0, v0 = cuda(sc["p_init"]), cuda(sc["v_init"])
    b = batch_of(api, sc)
    max_lane = int(np.diff(sc["lane_off"]).max())
    sig = tune.signature(max_lane, N, float(np.mean(sc["K"])), 1, kind="batch")
    path = str(tmp_path / "tune.json")
    ctx = api.Context()
    run = lambda c: api.batch_loss_grad(theta, p0, v0, b, Y, ctx=c)
    shape, how, timings = tune.tuned(ctx, run, max_lane, sig, repeats=2, path=path)
    assert how == "tuned" and len(timings) >= 4
    assert 32 * shape[0] * shape[1] >= max_lane
    assert ctx.tuning == tuple(shape)
    sl, tot, g, _, _ = run(ctx)
    ctx2 = api.Context()
    sl2, tot2, g2, _, _ = run(ctx2)                 # default shape
    torch.cuda.synchronize()
    assert ctx.check_status() == 0
    np.testing.assert_allclose(sl.cpu().numpy(), sl2.cpu().numpy(), rtol=1e-5, atol=1e-12)
    gn, g2n = g.double().cpu().numpy(), g2.double().cpu().numpy()
    np.testing.assert_allclose(gn, g2n, rtol=0, atol=1e-4 * np.abs(g2n).max())
    shape2, how2, _ = tune.tuned(api.Context(), run, max_lane, sig, path=path)
    assert how2 == "cache" and tuple(shape2) == tuple(shape)


@pytest.mark.parametrize("shape", [(0, 2, 1, 3, 8), (0, 4, 2, 8, 8), (0, 8, 2, 5, 8), (0, 0, 0, 64, 8)])
def test_batch_fit_single_launch_equals_graph(api, shape):
    """The batched fit as one persistent launch (scenarios with their own K,
    observation stride and segments, the forward skipped where a scenario's
    K fits the interval) against the per-iteration graph: loss history and
    per-scenario losses and parameters bit for bit."""
    sc, rng = small_batch(207, n_scen=9)
    Y = targets_for(sc, rng)
    N = int(sc["lane_off"][-1])
    th0 = synth.f32(sc["theta_true"] * np.r_[rng.uniform(0.8, 1.2, size=(5, N)), np.ones((1, N))])
    b = batch_of(api, sc)
    out = {}
    for mode in ("graph", "single"):
        ctx = api.Context(*shape)
        ctx.set_fit_mode(mode)
        th = cuda(th0)
        hist, sl = api.batch_fit(th, cuda(sc["p_init"]), cuda(sc["v_init"]), b, cuda(Y), 5, ctx=ctx)
        torch.cuda.synchronize()
        assert ctx.check_status() == 0 and ctx.last_fit_form() == mode
        out[mode] = (th.cpu().numpy(), hist.cpu().numpy(), sl.cpu().numpy())
    for q in range(3):
        np.testing.assert_array_equal(out["single"][q], out["graph"][q])
