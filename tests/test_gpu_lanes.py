"""GPU parity of the lane geometry and the training-free prediction pipeline
(paper Sec. IV-B, Sec. V-C) through the C-ABI against the FP64 oracle
(oracle/lanes.py plus the simulator oracle for the fit and the rollout).

Lane assignment is an argmin decided in FP32 on the GPU and FP64 in the
oracle: the scenes are checked (oracle side) to have no point whose two
nearest lanes are within 1 cm, so the decision is unique; then assignment and
the lane-sorted order are compared bit for bit.  Arc lengths and positions:
1e-3 m.  Fitted parameters: as the fit parity tests (rtol 1e-4)."""
import numpy as np
import pytest

import oracle
from oracle import lanes as G
from paper_2412_16750_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A_MIN = -10.0


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16750_gb300 import api as _api
    return _api


def cuda(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def polylines(sc):
    o = sc["pt_off"]
    return [np.stack([sc["px"][a:b], sc["py"][a:b]], axis=1).astype(np.float64) for a, b in zip(o[:-1], o[1:])]


def oracle_assign(sc, polys, frame, cols):
    """(lane, s, d, margin) at one frame for the agents cols (margin: second
    nearest minus nearest distance)."""
    out = []
    for i in cols:
        q = (float(sc["x"][frame, i]), float(sc["y"][frame, i]))
        dists = []
        for l in range(sc["lane_lo"][i], sc["lane_hi"][i]):
            s, d, dist = G.project(polys[l], q)
            dists.append((dist, l, s, d))
        dists.sort(key=lambda t: (t[0], t[1]))
        margin = dists[1][0] - dists[0][0] if len(dists) > 1 else np.inf
        out.append((dists[0][1], dists[0][2], dists[0][3], margin))
    return out


def small_scene(seed, n_scen=30):
    return synth.prediction_scenes(n_scen, np.random.default_rng(seed))


def lanes_of(api, sc):
    return api.Lanes(cuda(sc["pt_off"], torch.int32), cuda(sc["px"]), cuda(sc["py"]))


def test_prepare_and_project_parity(api):
    sc = small_scene(3)
    polys = polylines(sc)
    L = lanes_of(api, sc)
    torch.cuda.synchronize()
    cum = np.concatenate([G.cumlen(p) for p in polys])
    np.testing.assert_allclose(L.lane_len.cpu().numpy(), cum, rtol=0, atol=1e-4)
    N = sc["x"].shape[1]
    H = sc["n_hist"]
    ref = oracle_assign(sc, polys, H - 1, range(N))
    assert min(r[3] for r in ref) > 1e-2, "choose a scene without near-tied lanes"
    lane, s, d = L.project(cuda(sc["x"][H - 1]), cuda(sc["y"][H - 1]), cuda(sc["lane_lo"], torch.int32),
                           cuda(sc["lane_hi"], torch.int32))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lane.cpu().numpy().ravel(), [r[0] for r in ref])
    np.testing.assert_allclose(s.cpu().numpy().ravel(), [r[1] for r in ref], rtol=0, atol=1e-3)
    np.testing.assert_allclose(d.cpu().numpy().ravel(), [r[2] for r in ref], rtol=0, atol=1e-3)
    # every history frame onto the assigned lane (fixed-lane mode)
    lane_g = lane.view(-1)
    _, s_all, d_all = L.project(cuda(sc["x"][:H]), cuda(sc["y"][:H]), lane_g, None)
    torch.cuda.synchronize()
    s_all, d_all = s_all.cpu().numpy(), d_all.cpu().numpy()
    for f in (0, 5, H - 1):
        for i in range(0, N, 7):
            sr, dr, _ = G.project(polys[ref[i][0]], (float(sc["x"][f, i]), float(sc["y"][f, i])))
            assert abs(s_all[f, i] - sr) < 1e-3 and abs(d_all[f, i] - dr) < 1e-3
    assert api.default_context().check_status() == 0


def test_unproject_parity(api):
    sc = small_scene(2)
    polys = polylines(sc)
    L = lanes_of(api, sc)
    rng = np.random.default_rng(3)
    R, C = 7, 64
    lane = rng.integers(0, sc["n_lanes"], size=C).astype(np.int32)
    s = synth.f32(rng.uniform(-20.0, 320.0, size=(R, C)))          # includes both extrapolations
    s[0, :4] = [0.0, 300.0, -1e-3, 2.0]                              # at the ends and on a point
    x, y = L.unproject(cuda(s), cuda(lane, torch.int32))
    torch.cuda.synchronize()
    x, y = x.cpu().numpy(), y.cpu().numpy()
    for r in range(R):
        for c in range(C):
            p = G.unproject(polys[lane[c]], float(s[r, c]))
            assert abs(x[r, c] - p[0]) < 1e-3 and abs(y[r, c] - p[1]) < 1e-3, (r, c)


def test_rollout_state_and_displacement(api):
    rng = np.random.default_rng(4)
    s = synth.f32(np.cumsum(rng.uniform(-0.2, 1.5, size=(11, 300)), axis=0))
    p, v = api.rollout_state(cuda(s), 9, 10, 0.1)
    pr, vr = G.rollout_state(s, 9, 10, float(np.float32(0.1)))
    np.testing.assert_allclose(p.cpu().numpy(), pr, atol=0)
    np.testing.assert_allclose(v.cpu().numpy(), vr, rtol=1e-5, atol=1e-4)
    F, N = 80, 1000
    px, py = synth.f32(rng.normal(0, 3, (F, N))), synth.f32(rng.normal(0, 3, (F, N)))
    tx, ty = synth.f32(rng.normal(0, 3, (F, N))), synth.f32(rng.normal(0, 3, (F, N)))
    ade, fde, sums = api.displacement(cuda(px), cuda(py), cuda(tx), cuda(ty), 2.0)
    a_r, f_r, m_r, (ma, mf, mm) = G.displacement_metrics(np.stack([px, py], 2), np.stack([tx, ty], 2), 2.0)
    np.testing.assert_allclose(ade.cpu().numpy(), a_r, rtol=1e-5)
    np.testing.assert_allclose(fde.cpu().numpy(), f_r, rtol=1e-5)
    sums = sums.cpu().numpy()
    assert abs(sums[0] / N - ma) < 1e-5 * ma and abs(sums[1] / N - mf) < 1e-5 * mf
    unambiguous = np.abs(f_r - 2.0) > 1e-4
    assert sums[2] == m_r.sum() or not unambiguous.all()


def oracle_pipeline(api, sc, n_iter):
    """The prediction pipeline from the oracle's primitives."""
    polys = polylines(sc)
    H, Fn = sc["n_hist"], sc["n_fut"]
    N = sc["x"].shape[1]
    dt = sc["dt"]
    asg = oracle_assign(sc, polys, H - 1, range(N))
    lane = np.array([a[0] for a in asg], np.int32)
    s_hist = np.array([[G.project(polys[lane[i]], (float(sc["x"][f, i]), float(sc["y"][f, i])))[0]
                        for i in range(N)] for f in range(H)])
    perm, lane_off = oracle.layout(lane, s_hist[0], sc["n_lanes"])
    s_sorted = s_hist[:, perm]
    p0, v0 = G.rollout_state(s_sorted, 0, 1, dt)
    th0 = np.array(api.RECON_INIT)[:, None].repeat(N, 1)
    length = np.full(N, api.PRED_LENGTH)
    th, hist = oracle.fit(lane_off, length, th0, p0, v0, H - 1, dt, s_sorted[1:], 1, n_iter, 0.1, 0.01,
                          api.PRED_BOX_LO, api.PRED_BOX_HI, A_MIN)
    pr, vr = G.rollout_state(s_sorted, H - 2, H - 1, dt)
    P, _ = oracle.forward(lane_off, length, th, pr, vr, Fn, dt, A_MIN)
    lane_s = lane[perm]
    xy = np.array([[G.unproject(polys[lane_s[i]], P[f, i]) for i in range(N)] for f in range(1, Fn + 1)])
    true = np.stack([sc["x"][H:, perm], sc["y"][H:, perm]], axis=2)
    ade, fde, miss, means = G.displacement_metrics(xy, true, 2.0)
    return dict(lane=lane, perm=perm, s_sorted=s_sorted, theta=th, hist=hist, xy=xy, ade=ade, fde=fde,
                margin=min(a[3] for a in asg))


def test_prediction_pipeline_parity(api):
    sc = small_scene(5, n_scen=12)
    n_iter = 5
    ref = oracle_pipeline(api, sc, n_iter)
    assert ref["margin"] > 1e-2
    H = sc["n_hist"]
    L = lanes_of(api, sc)
    out = api.predict_rollout(L, cuda(sc["x"][:H]), cuda(sc["y"][:H]), cuda(sc["lane_lo"], torch.int32),
                              cuda(sc["lane_hi"], torch.int32), sc["dt"], sc["n_fut"], n_iter)
    torch.cuda.synchronize()
    perm = out["perm"].cpu().numpy()
    np.testing.assert_array_equal(perm, ref["perm"])
    np.testing.assert_array_equal(out["lane"].cpu().numpy(), ref["lane"][ref["perm"]])
    np.testing.assert_allclose(out["s_hist"].cpu().numpy(), ref["s_sorted"], rtol=0, atol=1e-3)
    np.testing.assert_allclose(out["loss"].cpu().numpy(), ref["hist"], rtol=1e-4)
    np.testing.assert_allclose(out["theta"].double().cpu().numpy(), ref["theta"], rtol=1e-4, atol=1e-4)
    xy = np.stack([out["x"].cpu().numpy(), out["y"].cpu().numpy()], axis=2)
    np.testing.assert_allclose(xy, ref["xy"], rtol=0, atol=2e-2)
    tx = cuda(sc["x"][H:, perm])
    ty = cuda(sc["y"][H:, perm])
    ade, fde, sums = api.displacement(out["x"], out["y"], tx, ty, 2.0)
    np.testing.assert_allclose(ade.cpu().numpy(), ref["ade"], rtol=0, atol=2e-2)
    np.testing.assert_allclose(fde.cpu().numpy(), ref["fde"], rtol=0, atol=2e-2)
    assert api.default_context().check_status() == 0


def test_bad_lane_index_sets_status(api):
    from paper_2412_16750_gb300 import lib
    sc = small_scene(6, n_scen=3)
    ctx = api.Context()
    L = api.Lanes(cuda(sc["pt_off"], torch.int32), cuda(sc["px"]), cuda(sc["py"]), ctx=ctx)
    bad = cuda(np.array([0, sc["n_lanes"] + 3], np.int32), torch.int32)
    x, y = L.unproject(cuda(np.array([1.0, 2.0])), bad)
    torch.cuda.synchronize()
    assert np.isnan(x.cpu().numpy()[0, 1])
    rc, flags = ctx.status()
    assert rc == lib.IDM_ERR_LANES and flags & lib.IDM_STATUS_BAD_LANES
    assert ctx.status()[0] == lib.IDM_OK


def test_full_size_prediction_sampled_lanes(api):
    """The prediction workload of the benchmark (10,000 scenarios) through
    the GPU pipeline; 40 sampled lanes (every agent on them) re-run by the
    oracle's pipeline: assignment, projected history, fitted parameters (5
    Adam iterations), rollout positions.  Lanes whose agents have near-tied
    nearest lanes are not sampled."""
    sc = synth.prediction_scenes(10000, np.random.default_rng(synth.SEED_BASE + 70))
    H, Fn = sc["n_hist"], sc["n_fut"]
    N = sc["x"].shape[1]
    n_iter = 5
    L = lanes_of(api, sc)
    out = api.predict_rollout(L, cuda(sc["x"][:H]), cuda(sc["y"][:H]), cuda(sc["lane_lo"], torch.int32),
                              cuda(sc["lane_hi"], torch.int32), sc["dt"], Fn, n_iter)
    torch.cuda.synchronize()
    perm = out["perm"].cpu().numpy()
    lane_off = out["lane_off"].cpu().numpy()
    s_g = out["s_hist"].cpu().numpy()
    th_g = out["theta"].double().cpu().numpy()
    x_g, y_g = out["x"].cpu().numpy(), out["y"].cpu().numpy()
    polys = polylines(sc)
    rng = np.random.default_rng(90)
    used = np.where(np.diff(lane_off) > 0)[0]
    checked = 0
    for l in rng.permutation(used):
        a0, a1 = lane_off[l], lane_off[l + 1]
        agents = perm[a0:a1]
        asg = oracle_assign(sc, polys, H - 1, agents)
        if min(x[3] for x in asg) < 1e-2 or any(x[0] != l for x in asg):
            continue
        # oracle pipeline on this lane alone (lanes do not interact)
        s_hist = np.array([[G.project(polys[l], (float(sc["x"][f, i]), float(sc["y"][f, i])))[0] for i in agents]
                           for f in range(H)])
        sub_perm, sub_off = oracle.layout(np.zeros(len(agents), np.int32), s_hist[0], 1)
        np.testing.assert_array_equal(agents[sub_perm], agents)      # the GPU's lane order
        np.testing.assert_allclose(s_g[:, a0:a1], s_hist, rtol=0, atol=1e-3)
        n = len(agents)
        p0, v0 = G.rollout_state(s_hist, 0, 1, sc["dt"])
        th0 = np.array(api.RECON_INIT)[:, None].repeat(n, 1)
        th, _ = oracle.fit(np.array([0, n], np.int32), np.full(n, api.PRED_LENGTH), th0, p0, v0, H - 1, sc["dt"],
                           s_hist[1:], 1, n_iter, 0.1, 0.01, api.PRED_BOX_LO, api.PRED_BOX_HI, A_MIN)
        np.testing.assert_allclose(th_g[:, a0:a1], th, rtol=1e-4, atol=1e-4)
        pr, vr = G.rollout_state(s_hist, H - 2, H - 1, sc["dt"])
        P, _ = oracle.forward(np.array([0, n], np.int32), np.full(n, api.PRED_LENGTH), th, pr, vr, Fn, sc["dt"], A_MIN)
        for j in range(n):
            for f in (0, Fn // 2, Fn - 1):
                p = G.unproject(polys[l], P[f + 1, j])
                assert abs(x_g[f, a0 + j] - p[0]) < 2e-2 and abs(y_g[f, a0 + j] - p[1]) < 2e-2
        checked += 1
        if checked == 40:
            break
    assert checked == 40
    assert api.default_context().check_status() == 0
