"""GPU parity of the single-trajectory filtering / reconstruction mode
(paper Sec. IV-A, settings and metrics of Sec. V-B) through the C-ABI
against the FP64 oracle (oracle/recon_oracle.c).

Tolerances: integer work (nearest steps, horizons) bit-exact; positions
within 1e-3 m; loss relative 1e-6; gradients: per parameter and for the
dp / dv fields, ||g - g_ref|| / ||g_ref|| <= 1e-4 and every element within
1e-3 * max |g_ref|.  The absolute-error seeds are signs, decided in FP32 on
the GPU and FP64 in the oracle: the inputs are built (from oracle values
only) so that no residual lies within 1e-2 m of zero, where the two could
disagree.
"""
import numpy as np
import pytest

from oracle import recon as R
from paper_2412_16750_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A_MIN = -10.0
F32 = lambda x: float(np.float32(x))  # noqa: E731


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16750_gb300 import api as _api
    return _api


def cuda(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def make_case(seed, n, dur, dt, dense=None, gap_min=1.0, noise=0.5, sort=True):
    rng = np.random.default_rng(seed)
    off, t, p = synth.recon_observations(n, dur, rng, dense=dense, gap_min=gap_min, gap_mean_extra=1.0,
                                        noise=noise, sort=sort)
    return dict(off=off, t=t, p=p, dt=F32(dt))


def oracle_setup(case):
    obs_k = R.nearest_steps(case["t"], case["dt"])
    K = R.horizons(case["off"], obs_k)
    p0, v0 = R.init_state(case["off"], case["t"], case["p"])
    return obs_k, K, synth.f32(p0), synth.f32(v0)


def leader_vars(rng, k_max, N):
    """A virtual leader near the paper's start (dp 10, dv 0), perturbed."""
    dp = synth.f32(10.0 + rng.uniform(-5.0, 20.0, size=(k_max, N)))
    dv = synth.f32(rng.uniform(-2.0, 2.0, size=(k_max, N)))
    return dp, dv


def param_vars(rng, N):
    lo, hi = (25.0, 0.8, 1.5, 5.0, 1.0), (40.0, 2.0, 4.0, 10.0, 3.0)
    th = np.vstack([rng.uniform(lo[q], hi[q], N) for q in range(5)] + [np.full(N, 4.0)])
    return synth.f32(th)


def drop_ambiguous(case, obs_k, K, th, dp, dv, p0, v0, margin=1e-2):
    """Remove observations whose oracle residual lies within margin of zero
    (their sign may differ between FP32 and FP64).  Oracle values only."""
    P, _, _ = R.forward(K, dp, dv, th, p0, v0, case["dt"], A_MIN)
    N = len(K)
    tr = np.repeat(np.arange(N), np.diff(case["off"]))
    r = P[np.minimum(obs_k, P.shape[0] - 1), tr] - case["p"]
    keep = (np.abs(r) >= margin) | (obs_k == 0)
    # keep every trajectory's first observation: it fixes the initial state
    keep[case["off"][:-1][np.diff(case["off"]) > 0]] = True
    counts = np.array([keep[case["off"][i]:case["off"][i + 1]].sum() for i in range(N)])
    off = np.zeros(N + 1, np.int32)
    off[1:] = np.cumsum(counts)
    out = dict(case, off=off, t=case["t"][keep], p=case["p"][keep])
    return out, obs_k[keep]


class GpuCase:
    """A Recon object whose initial state is overridden with the oracle's
    (float32-rounded) values, so both sides start identically."""

    def __init__(self, api, case, p0, v0):
        self.r = api.Recon(cuda(case["off"], torch.int32), cuda(case["t"]), cuda(case["p"]), case["dt"], A_MIN)
        self.r.p_init.copy_(cuda(p0))
        self.r.v_init.copy_(cuda(v0))


def grad_close(g, ref, rtol=1e-4, elem=1e-3, what=""):
    nr = np.linalg.norm(ref)
    if nr == 0.0:
        assert np.max(np.abs(g)) == 0.0, what
        return
    err = np.linalg.norm(g - ref) / nr
    assert err <= rtol, "%s: relative error %.3g" % (what, err)
    assert np.max(np.abs(g - ref)) <= elem * np.max(np.abs(ref)), what


CASES = [
    # (seed, n, duration range s, dt, dense sampling, min gap) -- dense
    # filtering, sparse reconstruction, several observations per step (5 and
    # 10, the second exercises the scan past 7)
    ("filter", 11, 70, (3.0, 30.0), 0.1, 0.1, 1.0),
    ("recon", 12, 70, (20.0, 240.0), 1.0, None, 1.0),
    ("multi5", 13, 45, (3.0, 20.0), 0.5, 0.1, 1.0),
    ("multi10", 14, 40, (3.0, 20.0), 1.0, 0.1, 1.0),
]


@pytest.mark.parametrize("name,seed,n,dur,dt,dense,gap", CASES)
def test_prepare_bitexact(api, name, seed, n, dur, dt, dense, gap):
    case = make_case(seed, n, dur, dt, dense, gap)
    obs_k, K, p0, v0 = oracle_setup(case)
    g = GpuCase(api, case, p0, v0).r
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g.obs_k.cpu().numpy()[:len(obs_k)], obs_k)
    np.testing.assert_array_equal(g.K.cpu().numpy()[:n], K)
    assert g.k_max == int(K.max())
    # the initial state in FP32 against the FP64 rule
    r = api.Recon(cuda(case["off"], torch.int32), cuda(case["t"]), cuda(case["p"]), case["dt"], A_MIN)
    p0r, v0r = R.init_state(case["off"], case["t"], case["p"])
    np.testing.assert_allclose(r.p_init.cpu().numpy()[:n], p0r, rtol=0, atol=0)
    np.testing.assert_allclose(r.v_init.cpu().numpy()[:n], v0r, rtol=2e-6, atol=1e-6)
    assert api.default_context().check_status() == 0


def test_prepare_ties_and_degenerate(api):
    # timestamps exactly half way between steps (binary dt) go to the later
    # step; a trajectory with one observation has K = 0 and v_init = 0; an
    # empty trajectory is allowed
    dt = 0.125
    t = np.array([0.0, 0.0625, 0.1875, 0.3125, 0.0, 0.0, 0.5, 0.5, 1.0625])
    p = np.array([0.0, 1.0, 2.0, 3.0, 7.0, 5.0, 6.0, 4.0, 9.0])
    off = np.array([0, 4, 5, 5, 9], np.int32)
    case = dict(off=off, t=t, p=p, dt=dt)
    obs_k, K, p0, v0 = oracle_setup(case)
    r = api.Recon(cuda(off, torch.int32), cuda(t), cuda(p), dt, A_MIN)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(r.obs_k.cpu().numpy(), obs_k)
    np.testing.assert_array_equal(obs_k[:4], [0, 1, 2, 3])
    np.testing.assert_array_equal(r.K.cpu().numpy(), K)
    np.testing.assert_array_equal(K, [3, 0, 0, 9])
    np.testing.assert_array_equal(r.v_init.cpu().numpy(), synth.f32(v0))
    np.testing.assert_array_equal(r.p_init.cpu().numpy(), synth.f32(p0))


@pytest.mark.parametrize("name,seed,n,dur,dt,dense,gap", CASES[:2])
def test_forward_parity(api, name, seed, n, dur, dt, dense, gap):
    case = make_case(seed, n, dur, dt, dense, gap)
    obs_k, K, p0, v0 = oracle_setup(case)
    rng = np.random.default_rng(seed + 100)
    k_max = int(K.max())
    dp, dv = leader_vars(rng, k_max, n)
    th = param_vars(rng, n)
    th[5, :5] = 3.0     # one warp with a non-integer power path
    g = GpuCase(api, case, p0, v0).r
    P, V, A = g.forward(cuda(th), cuda(dp), cuda(dv))
    torch.cuda.synchronize()
    Pr, Vr, Ar = R.forward(K, dp, dv, th, p0, v0, case["dt"], A_MIN)
    np.testing.assert_allclose(P.double().cpu().numpy(), Pr, rtol=0, atol=1e-3)
    np.testing.assert_allclose(V.double().cpu().numpy(), Vr, rtol=0, atol=1e-4)
    np.testing.assert_allclose(A.double().cpu().numpy(), Ar, rtol=0, atol=1e-3)


@pytest.mark.parametrize("name,seed,n,dur,dt,dense,gap", CASES)
def test_loss_grad_parity(api, name, seed, n, dur, dt, dense, gap):
    case = make_case(seed, n, dur, dt, dense, gap)
    obs_k, K, p0, v0 = oracle_setup(case)
    rng = np.random.default_rng(seed + 200)
    k_max = int(K.max())
    dp, dv = leader_vars(rng, k_max, n)
    th = param_vars(rng, n)
    case, obs_k = drop_ambiguous(case, obs_k, K, th, dp, dv, p0, v0)
    K = R.horizons(case["off"], obs_k)          # a dropped last observation shortens K
    dp, dv = dp[:int(K.max())], dv[:int(K.max())]
    P, V, _ = R.forward(K, dp, dv, th, p0, v0, case["dt"], A_MIN)
    L, gP = R.mae_seed(K, case["off"], obs_k, case["p"], P)
    gr, gdp, gdv, gp0, gv0 = R.adjoint(K, dp, dv, th, case["dt"], V, gP, A_MIN)

    g = GpuCase(api, case, p0, v0).r
    loss, gth, gdp_g, gdv_g, gp_g, gv_g = g.loss_grad(cuda(th), cuda(dp), cuda(dv))
    torch.cuda.synchronize()
    assert abs(loss.item() - L) <= 1e-6 * L
    gth = gth.double().cpu().numpy()
    for q in range(6):
        grad_close(gth[q], gr[q], what="param %d" % q)
    grad_close(gdp_g.double().cpu().numpy(), gdp, what="dp")
    grad_close(gdv_g.double().cpu().numpy(), gdv, what="dv")
    grad_close(gp_g.double().cpu().numpy(), gp0, what="p_init")
    grad_close(gv_g.double().cpu().numpy(), gv0, what="v_init")
    assert api.default_context().check_status() == 0


def _iterate_residuals(case, obs_k, K, th, dp, dv, p0, v0, n_iter, lo, hi):
    """|residual| of every observation at each of the n_iter iterates of the
    fit, replayed with the oracle's primitives (forward, seeds, adjoint) and
    the Adam rule of the fit; used only to choose unambiguous inputs."""
    n = len(K)
    th, dp, dv = th.astype(np.float64).copy(), dp.astype(np.float64).copy(), dv.astype(np.float64).copy()
    mt, vt = np.zeros((5, n)), np.zeros((5, n))
    mp, vp, mv, vv = (np.zeros_like(dp) for _ in range(4))
    tr = np.repeat(np.arange(n), np.diff(case["off"]))
    out = []
    for it in range(n_iter):
        P, V, _ = R.forward(K, dp, dv, th, p0, v0, case["dt"], A_MIN)
        out.append(np.abs(P[obs_k, tr] - case["p"]))
        _, gP = R.mae_seed(K, case["off"], obs_k, case["p"], P)
        g, gdp, gdv, _, _ = R.adjoint(K, dp, dv, th, case["dt"], V, gP, A_MIN)
        lr = 0.1 + (0.01 - 0.1) * it / max(n_iter - 1, 1)
        t = it + 1

        def adam(x, gg, m, v):
            m[:] = 0.9 * m + 0.1 * gg
            v[:] = 0.999 * v + 0.001 * gg * gg
            return x - lr * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
        th[:5] = np.clip(adam(th[:5], g[:5], mt, vt), np.array(lo)[:, None], np.array(hi)[:, None])
        dp = adam(dp, gdp, mp, vp)
        dv = adam(dv, gdv, mv, vv)
    return out


def test_fit_parity(api):
    case = make_case(21, 70, (5.0, 40.0), 0.1, 0.1, 1.0)
    obs_k, K, p0, v0 = oracle_setup(case)
    n = 70
    k_max = int(K.max())
    th = synth.f32(np.array(api.RECON_INIT)[:, None].repeat(n, 1))
    dp = np.full((k_max, n), 10.0)
    dv = np.zeros((k_max, n))
    lo, hi = api.RECON_BOX_LO, api.RECON_BOX_HI
    n_iter = 4
    # residual signs must not be ambiguous at any iterate: drop observations
    # that come within 1e-2 m of the oracle's trajectory (oracle values only)
    for _ in range(4):
        res = _iterate_residuals(case, obs_k, K, th, dp, dv, p0, v0, n_iter, lo, hi)
        amb = np.any([(r < 1e-2) for r in res], axis=0) & (obs_k > 0)
        if not amb.any():
            break
        keep = ~amb
        counts = np.array([keep[case["off"][i]:case["off"][i + 1]].sum() for i in range(n)])
        off = np.zeros(n + 1, np.int32)
        off[1:] = np.cumsum(counts)
        case = dict(case, off=off, t=case["t"][keep], p=case["p"][keep])
        obs_k = obs_k[keep]
    assert not amb.any()
    K = R.horizons(case["off"], obs_k)
    k_max = int(K.max())
    dp, dv = dp[:k_max], dv[:k_max]
    th_r, dp_r, dv_r, hist_r = R.fit(K, dp, dv, th, p0, v0, case["dt"], case["off"], obs_k, case["p"], n_iter,
                                     0.1, 0.01, lo, hi, A_MIN)

    g = GpuCase(api, case, p0, v0).r
    assert g.k_max == k_max
    th_g, dp_g, dv_g = cuda(th), cuda(dp), cuda(dv)
    hist = g.fit(th_g, dp_g, dv_g, n_iter, 0.1, 0.01, lo, hi)
    torch.cuda.synchronize()
    np.testing.assert_allclose(hist.cpu().numpy(), hist_r, rtol=1e-5)
    np.testing.assert_allclose(th_g.double().cpu().numpy(), th_r, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(dp_g.double().cpu().numpy(), dp_r, rtol=0, atol=1e-3)
    np.testing.assert_allclose(dv_g.double().cpu().numpy(), dv_r, rtol=0, atol=1e-3)


def test_metrics_parity(api):
    case = make_case(31, 70, (20.0, 200.0), 1.0, None, 1.0)
    obs_k, K, p0, v0 = oracle_setup(case)
    rng = np.random.default_rng(310)
    k_max = int(K.max())
    dp, dv = leader_vars(rng, k_max, 70)
    th = param_vars(rng, 70)
    P, _, A = R.forward(K, dp, dv, th, p0, v0, case["dt"], A_MIN)
    ref = R.metrics(K, case["off"], obs_k, case["p"], P, A)
    g = GpuCase(api, case, p0, v0).r
    out = g.metrics(cuda(th), cuda(dp), cuda(dv)).cpu().numpy()
    np.testing.assert_allclose(out[:3], ref[:3], rtol=1e-5)
    assert out[3] == ref[3]


def test_argument_errors(api):
    from paper_2412_16750_gb300 import lib
    case = make_case(41, 8, (3.0, 6.0), 0.1, 0.1, 1.0)
    g = api.Recon(cuda(case["off"], torch.int32), cuda(case["t"]), cuda(case["p"]), case["dt"], A_MIN)
    th, dp, dv = g.init_vars()
    rec = g.c()
    rec.ld = g.N - 1
    with pytest.raises(lib.IdmError) as e:
        lib.idm_recon_forward(g.ctx.handle, rec, lib.make_params(th), dp, dv)
    assert e.value.code == lib.IDM_ERR_ARG
    rec = g.c()
    rec.dt = 0.0
    with pytest.raises(lib.IdmError):
        lib.idm_recon_loss_grad(g.ctx.handle, rec, lib.make_params(th), dp, dv)
    with pytest.raises(lib.IdmError):
        lib.idm_recon_fit(g.ctx.handle, g.c(), lib.make_params(th), dp, dv, 0, 0.1, 0.01, api.RECON_BOX_LO,
                          api.RECON_BOX_HI)


def test_device_status_bad_observations(api):
    from paper_2412_16750_gb300 import lib
    # decreasing timestamps inside a trajectory: reported, nothing out of bounds
    off = np.array([0, 3, 6], np.int32)
    t = np.array([0.0, 0.5, 0.3, 0.0, 0.2, 0.4])
    p = np.arange(6, dtype=np.float64)
    ctx = api.Context()
    api.Recon(cuda(off, torch.int32), cuda(t), cuda(p), 0.1, A_MIN, ctx=ctx)
    rc, flags = ctx.status()
    assert rc == lib.IDM_ERR_OBS and flags & lib.IDM_STATUS_BAD_OBS
    # a horizon beyond k_max
    case = make_case(42, 8, (3.0, 6.0), 0.1, 0.1, 1.0)
    g = api.Recon(cuda(case["off"], torch.int32), cuda(case["t"]), cuda(case["p"]), case["dt"], A_MIN, ctx=ctx)
    th, dp, dv = g.init_vars()
    g.K[0] = g.k_max + 5
    g.loss_grad(th, dp, dv)
    rc, flags = ctx.status()
    assert rc == lib.IDM_ERR_OBS
    assert ctx.status()[0] == lib.IDM_OK


def test_full_size_reconstruction_workload(api):
    """The reconstruction workload (21,750 trajectories, sampling intervals
    >= 1 s, up to 20 min, dt = 1 s) in the launch the benchmark times: the
    loss and every gradient against the oracle over all trajectories whose
    residuals are unambiguous (the FP64 oracle runs the whole set)."""
    spec = synth.RECON_SPEC
    case = make_case(synth.SEED_BASE + 77, spec["n"], spec["dur"], spec["dt"], None, spec["gap_min"],
                     spec["noise"])
    obs_k, K, p0, v0 = oracle_setup(case)
    n = spec["n"]
    k_max = int(K.max())
    th = synth.f32(np.array(api.RECON_INIT)[:, None].repeat(n, 1))
    dp = np.full((k_max, n), 10.0, np.float32)
    dv = np.zeros((k_max, n), np.float32)
    P, V, _ = R.forward(K, dp, dv, th, p0, v0, case["dt"], A_MIN)
    L, gP = R.mae_seed(K, case["off"], obs_k, case["p"], P)
    gr, gdp, gdv, _, _ = R.adjoint(K, dp, dv, th, case["dt"], V, gP, A_MIN)
    tr = np.repeat(np.arange(n), np.diff(case["off"]))
    res = np.abs(P[obs_k, tr] - case["p"])
    amb = np.zeros(n, bool)
    np.logical_or.at(amb, tr, (res < 1e-2) & (obs_k > 0))
    del P, V, gP

    g = GpuCase(api, case, p0, v0).r
    loss, gth, gdp_g, gdv_g, _, _ = g.loss_grad(cuda(th), cuda(dp), cuda(dv))
    torch.cuda.synchronize()
    assert abs(loss.item() - L) <= 1e-6 * L
    ok = ~amb
    assert ok.mean() > 0.9
    gth = gth.double().cpu().numpy()
    for q in range(5):
        grad_close(gth[q][ok], gr[q][ok], what="param %d" % q)
    grad_close(gdp_g.double().cpu().numpy()[:, ok], gdp[:, ok], what="dp")
    grad_close(gdv_g.double().cpu().numpy()[:, ok], gdv[:, ok], what="dv")
    assert api.default_context().check_status() == 0


def test_padded_row_stride(api):
    """Per-step arrays with a row stride larger than the trajectory count
    (ld > N): the same loss and gradients as the packed layout."""
    from paper_2412_16750_gb300 import lib
    case = make_case(51, 45, (3.0, 25.0), 0.1, 0.1, 1.0)
    obs_k, K, p0, v0 = oracle_setup(case)
    rng = np.random.default_rng(510)
    k_max, n = int(K.max()), 45
    dp, dv = leader_vars(rng, k_max, n)
    th = param_vars(rng, n)
    case, obs_k = drop_ambiguous(case, obs_k, K, th, dp, dv, p0, v0)
    K = R.horizons(case["off"], obs_k)
    dp, dv = dp[:int(K.max())], dv[:int(K.max())]
    g = GpuCase(api, case, p0, v0).r
    loss_a, gth_a, gdp_a, gdv_a, _, _ = g.loss_grad(cuda(th), cuda(dp), cuda(dv))
    ld = 77
    dp_p = np.full((g.k_max, ld), np.nan, np.float32)
    dv_p = np.full((g.k_max, ld), np.nan, np.float32)
    dp_p[:, :n], dv_p[:, :n] = dp, dv
    rec = g.c()
    rec.ld = ld
    loss = torch.zeros((), device="cuda", dtype=torch.float64)
    gth = torch.empty((6, n), device="cuda")
    gdp = torch.full((g.k_max, ld), 7.0, device="cuda")
    gdv = torch.full((g.k_max, ld), 7.0, device="cuda")
    dpt, dvt, tht = cuda(dp_p), cuda(dv_p), cuda(th)
    lib.idm_recon_loss_grad(g.ctx.handle, rec, lib.make_params(tht), dpt, dvt, loss, lib.make_params(gth), gdp, gdv)
    torch.cuda.synchronize()
    assert abs(loss.item() - loss_a.item()) <= 1e-12 * abs(loss_a.item())   # warp sums added in any order
    np.testing.assert_array_equal(gth.cpu().numpy(), gth_a.cpu().numpy())
    np.testing.assert_array_equal(gdp.cpu().numpy()[:, :n], gdp_a.cpu().numpy())
    np.testing.assert_array_equal(gdv.cpu().numpy()[:, :n], gdv_a.cpu().numpy())
    assert np.all(gdp.cpu().numpy()[:, n:] == 7.0)          # the padding is not written
    assert api.default_context().check_status() == 0


def test_edge_trajectories(api):
    """Degenerate and extreme trajectories in one call: no observation, a
    single observation (K = 0), several observations at step 0 only, every
    observation at one step (a step with 9 observations), a long trajectory
    (K = 3,000 at dt = 0.1 s), and a count (33) that leaves a one-lane tail
    warp: loss and every gradient against the oracle (the long trajectory
    with tolerances scaled to its FP32 drift)."""
    dt = F32(0.1)
    rng = np.random.default_rng(61)
    ts, ps, off = [], [], [0]

    def add(t, p):
        ts.append(np.asarray(t, np.float64)); ps.append(np.asarray(p, np.float64)); off.append(off[-1] + len(t))

    add([], [])                                            # no observation
    add([0.0], [5.0])                                      # a single observation
    add([0.0, 0.01, 0.02], [1.0, 1.2, 1.3])                # several at step 0 only
    add([0.0] + [0.96 + 0.01 * j for j in range(9)], [0.0] + list(8.0 + rng.uniform(-3, 3, 9)))   # 9 at step 10
    long_t = np.append(np.arange(0.0, 299.5, 0.7), 300.0)
    add(long_t, 12.0 * long_t + rng.normal(0, 2.0, len(long_t)))   # K = 3000
    for _ in range(28):
        T = rng.uniform(2.0, 8.0)
        t = np.arange(0.0, T, 0.3)
        add(t, rng.uniform(0, 50) + rng.uniform(5, 20) * t + rng.normal(0, 1.0, len(t)))
    case = dict(off=np.array(off, np.int32), t=synth.f32(np.concatenate(ts)), p=synth.f32(np.concatenate(ps)), dt=dt)
    n = len(off) - 1
    assert n == 33
    obs_k, K, p0, v0 = oracle_setup(case)
    assert K[0] == 0 and K[1] == 0 and K[2] == 0 and K[3] == 10 and K[4] == 3000
    k_max = int(K.max())
    dp, dv = leader_vars(rng, k_max, n)
    th = param_vars(rng, n)
    case, obs_k = drop_ambiguous(case, obs_k, K, th, dp, dv, p0, v0)
    K = R.horizons(case["off"], obs_k)
    assert K[4] == 3000 and K[3] == 10
    P, V, _ = R.forward(K, dp, dv, th, p0, v0, case["dt"], A_MIN)
    L, gP = R.mae_seed(K, case["off"], obs_k, case["p"], P)
    gr, gdp, gdv, gp0, gv0 = R.adjoint(K, dp, dv, th, case["dt"], V, gP, A_MIN)
    g = GpuCase(api, case, p0, v0).r
    np.testing.assert_array_equal(g.K.cpu().numpy()[:n], K)
    loss, gth, gdp_g, gdv_g, gp_g, gv_g = g.loss_grad(cuda(th), cuda(dp), cuda(dv))
    Pg, _, _ = g.forward(cuda(th), cuda(dp), cuda(dv))
    torch.cuda.synchronize()
    # positions: 1e-3 m over the first 100 steps; over 3,000 steps the FP32
    # speed drifts, bounded here by 1e-2 m (the loss moves by at most the
    # number of observations times that)
    Pg = Pg.double().cpu().numpy()
    assert np.max(np.abs(Pg[:101] - P[:101])) <= 1e-3
    drift = np.max(np.abs(Pg - P))
    assert drift <= 1e-2, drift
    n_obs_long = int(np.sum(obs_k[case["off"][4]:case["off"][5]] > 0))
    assert abs(loss.item() - L) <= 1e-6 * L + n_obs_long * drift
    gth = gth.double().cpu().numpy()
    short = np.array([i for i in range(n) if i != 4])
    for q in range(6):
        grad_close(gth[q][short], gr[q][short], what="param %d" % q)
        assert abs(gth[q][4] - gr[q][4]) <= 1e-3 * abs(gr[q][4]) + 1e-6, q    # the 3,000-step trajectory
    grad_close(gdp_g.double().cpu().numpy()[:, short], gdp[:, short], what="dp")
    grad_close(gdv_g.double().cpu().numpy()[:, short], gdv[:, short], what="dv")
    for gg, rr in ((gdp_g, gdp), (gdv_g, gdv)):
        col = gg.double().cpu().numpy()[:, 4]
        assert np.linalg.norm(col - rr[:, 4]) <= 1e-3 * np.linalg.norm(rr[:, 4])
    grad_close(gv_g.double().cpu().numpy()[short], gv0[short], what="v_init")
    # trajectories without steps have zero gradients everywhere
    for i in (0, 1, 2):
        assert np.all(gth[:, i] == 0.0)
    assert api.default_context().check_status() == 0
