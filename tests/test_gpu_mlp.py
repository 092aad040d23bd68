"""GPU parity of the learned initializer's tensor-core kernels against the
FP64 oracle (oracle/mlp_oracle.py), through the C-ABI.

Both sides use the same bf16-rounded weights and inputs; the GPU keeps bf16
activations and accumulates in FP32 on the tensor cores, so the bar is the
one stated for this part: outputs within 1e-2 (relative), weight gradients
with cosine >= 0.999 per tensor.  The plain GEMM is held much tighter (FP32
accumulation of exact bf16 products).
"""
import numpy as np
import pytest

import oracle
from oracle import mlp_oracle as M
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


def bf16_round(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def to_bf16_cuda(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to("cuda").contiguous()


def bf16_weights(w):
    """The bf16 values the kernels multiply with (biases stay FP32)."""
    d = M.unpack(np.asarray(w, dtype=np.float64).copy())
    for name in ("W1", "W2", "W3", "W4"):
        d[name] = bf16_round(d[name])
    return M.pack(d)


def cosine(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


# ---------------------------------------------------------------------------
# the GEMM building block
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M_,N_,K_", [(1, 16, 16), (128, 256, 80), (300, 80, 256), (1000, 16, 2048),
                                      (257, 512, 64), (130, 48, 208)])
def test_gemm_bf16(api, M_, N_, K_):
    from paper_2412_16750_gb300 import lib
    rng = np.random.default_rng(M_ * 7 + N_ + K_)
    A = rng.normal(size=(M_, K_))
    B = rng.normal(size=(N_, K_))
    At, Bt = to_bf16_cuda(A), to_bf16_cuda(B)
    C = torch.full((M_, N_), float("nan"), device="cuda", dtype=torch.float32)
    status = torch.zeros(1, device="cuda", dtype=torch.int32)
    assert lib.idm_gemm_bf16(At, Bt, M_, N_, K_, C, status) == lib.IDM_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Ab, Bb = At.double().cpu().numpy(), Bt.double().cpu().numpy()
    ref = Ab @ Bb.T
    bound = np.abs(Ab) @ np.abs(Bb).T
    err = np.abs(C.double().cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * bound + 1e-30), float((err / (bound + 1e-30)).max())


def test_gemm_bf16_rejects_bad_shapes(api):
    from paper_2412_16750_gb300 import lib
    A = torch.zeros((4, 32), device="cuda", dtype=torch.bfloat16)
    C = torch.zeros((4, 16), device="cuda", dtype=torch.float32)
    st = torch.zeros(1, device="cuda", dtype=torch.int32)
    assert lib.idm_gemm_bf16(A, A, 4, 8, 32, C, st) == lib.IDM_ERR_ARG     # N not a multiple of 16
    assert lib.idm_gemm_bf16(A, A, 4, 16, 24, C, st) == lib.IDM_ERR_ARG    # K not a multiple of 16
    assert lib.idm_gemm_bf16(A, A, 0, 16, 32, C, st) == lib.IDM_ERR_ARG
    assert lib.idm_gemm_bf16(A, A, 4, 16, 32, C, None) == lib.IDM_ERR_ARG


# ---------------------------------------------------------------------------
# network: forward, loss + gradient, Adam step
# ---------------------------------------------------------------------------

def random_batch(B, seed):
    rng = np.random.default_rng(seed)
    X = bf16_round(rng.normal(scale=0.7, size=(B, 80)))
    T = rng.uniform(0.05, 0.95, size=(B, 5))
    return X, T


@pytest.mark.parametrize("B", [1, 300, 1000])
def test_mlp_forward(api, B):
    w = synth.mlp_init(0)
    X, _ = random_batch(B, 10 + B)
    net = api.Mlp(max_batch=1024, weights=w)
    S = net.forward(to_bf16_cuda(X)).double().cpu().numpy()
    ref = M.forward(bf16_weights(w), X)["s"]
    np.testing.assert_allclose(S, ref, rtol=1e-2, atol=1e-3)
    assert net.status() == (0, 0)


@pytest.mark.parametrize("B", [130, 1000])
def test_mlp_loss_grad(api, B):
    w = synth.mlp_init(1)
    X, T = random_batch(B, 20 + B)
    net = api.Mlp(max_batch=1024, weights=w)
    loss, g = net.loss_grad(to_bf16_cuda(X), torch.as_tensor(T, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    L_ref, g_ref = M.loss_grad(bf16_weights(w), X, synth.f32(T))
    assert abs(loss.item() - L_ref) <= 1e-2 * L_ref
    gd, rd = M.unpack(g.double().cpu().numpy()), M.unpack(g_ref)
    for name, _ in M.SHAPES:
        c = cosine(gd[name], rd[name])
        assert c >= 0.999, (name, c)
        ratio = np.linalg.norm(gd[name]) / np.linalg.norm(rd[name])
        assert abs(ratio - 1) <= 0.02, (name, ratio)
    assert net.status() == (0, 0)


def test_mlp_train_step_matches_adam(api):
    w = synth.mlp_init(2)
    X, T = random_batch(512, 30)
    Xt, Tt = to_bf16_cuda(X), torch.as_tensor(T, dtype=torch.float32, device="cuda")
    net = api.Mlp(max_batch=512, weights=w)
    _, g_ref = M.loss_grad(bf16_weights(w), X, synth.f32(T))
    w_ref, _, _ = M.adam_step(w, g_ref, np.zeros_like(w), np.zeros_like(w), 1, 1e-3)
    net.train_step(Xt, Tt, 1e-3)
    w_gpu = net.get_weights().double().cpu().numpy()
    # first Adam step moves every weight by ~ lr sign(g): compare the updates
    c = cosine(w_gpu - w, w_ref - w)
    assert c >= 0.98, c
    # training on a fixed batch drives the loss down
    losses = [net.train_step(Xt, Tt, 1e-3).item() for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    assert net.status() == (0, 0)


def test_set_get_weights_roundtrip(api):
    w = synth.mlp_init(3)
    net = api.Mlp(max_batch=128, weights=w)
    np.testing.assert_array_equal(net.get_weights().cpu().numpy(), w.astype(np.float32))


# ---------------------------------------------------------------------------
# features and parameter prediction
# ---------------------------------------------------------------------------

def noisy_prefix_scene(n_lanes, per_lane, K, s, seed):
    rng = np.random.default_rng(seed)
    counts = [per_lane] * n_lanes
    sc = synth.make_scene(counts, rng)
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    n_obs = K // s
    Y = synth.f32(P[s::s][:n_obs] + rng.normal(0, 0.5, size=(n_obs, P.shape[1])))
    return sc, Y


def test_features_and_labels(api):
    sc, Y = noisy_prefix_scene(7, 23, 44, 2, 40)
    N = int(sc["lane_off"][-1])
    perm = np.random.default_rng(41).permutation(N)[:150].astype(np.int32)
    scene = api.Scene.from_lane_off(torch.as_tensor(sc["lane_off"]), torch.as_tensor(sc["length"]))
    th = torch.as_tensor(sc["theta_true"], dtype=torch.float32, device="cuda").contiguous()
    X, lab = api.mlp_features(scene, torch.as_tensor(sc["p_init"]), torch.as_tensor(sc["v_init"]), 44, DT,
                              torch.as_tensor(Y), 2, perm=torch.as_tensor(perm), theta=th)
    Xr = M.features(sc["lane_off"], sc["p_init"], sc["v_init"], Y, 2, DT, perm=perm)
    Xg = X.double().cpu().numpy()
    # the GPU rounds its FP32 feature to bf16: within one bf16 step of the exact value
    np.testing.assert_allclose(Xg, Xr, rtol=2.0 ** -8, atol=1e-6)
    Lr = M.labels(sc["theta_true"], synth.BOX_LO, synth.BOX_HI, perm=perm)
    np.testing.assert_allclose(lab.double().cpu().numpy(), Lr, rtol=1e-5, atol=1e-6)


def test_predict_params_maps_into_the_box(api):
    w = synth.mlp_init(4) * 2.0
    X, _ = random_batch(700, 50)
    net = api.Mlp(max_batch=256, weights=w)          # 700 rows: three chunks of max_batch
    th = torch.zeros((6, 700), device="cuda", dtype=torch.float32)
    th[5] = 4.0
    net.predict_params(to_bf16_cuda(X), th)
    got = th.double().cpu().numpy()
    ref = M.predict_params(bf16_weights(w), X, synth.BOX_LO, synth.BOX_HI)
    width = (np.array(synth.BOX_HI) - np.array(synth.BOX_LO))[:, None]
    assert np.max(np.abs(got[:5] - ref) / width) <= 1e-2
    assert np.all(got[5] == 4.0)
    for q in range(5):
        assert synth.BOX_LO[q] <= got[q].min() and got[q].max() <= synth.BOX_HI[q]


# ---------------------------------------------------------------------------
# what the trained network gains over the plain initial guess
# ---------------------------------------------------------------------------

def test_learned_init_beats_plain(api):
    """Train the network on simulated prefixes, then fit a held-out scene from
    the learned and from the plain initial guess with the same Adam schedule;
    the FP64 oracle scores both fits against the noise-free truth."""
    # training set: 300K vehicles, 20-step noisy prefixes, shuffled
    rng = np.random.default_rng(60)
    tr = synth.make_scene([100] * 3000, rng)
    N = int(tr["lane_off"][-1])
    scene = api.Scene.from_lane_off(torch.as_tensor(tr["lane_off"]), torch.as_tensor(tr["length"]))
    th = torch.as_tensor(tr["theta_true"], dtype=torch.float32, device="cuda").contiguous()
    P = api.simulate(th, torch.as_tensor(tr["p_init"]), torch.as_tensor(tr["v_init"]), scene, 20, DT)
    Y = P[1:] + torch.as_tensor(rng.normal(0, 0.5, size=(20, N)), dtype=torch.float32, device="cuda")
    perm = torch.as_tensor(rng.permutation(N).astype(np.int32))
    X, lab = api.mlp_features(scene, torch.as_tensor(tr["p_init"]), torch.as_tensor(tr["v_init"]), 20, DT, Y,
                              1, perm=perm, theta=th)
    net = api.Mlp(max_batch=4096, weights=synth.mlp_init(0))
    hist = net.train(X, lab, 4096, 600, 2e-3, 2e-4).cpu().numpy()
    assert net.status() == (0, 0)
    assert hist[-20:].mean() < 0.5 * hist[:20].mean()

    # held-out scene: 10 lanes x 100 vehicles, 100 steps, every step observed
    sc = synth.config0()
    K = sc["K"]
    Pc, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    clean = Pc[1:K + 1]
    Yh = synth.f32(clean + np.random.default_rng(61).normal(0, 0.5, size=clean.shape))
    sch = api.Scene.from_lane_off(torch.as_tensor(sc["lane_off"]), torch.as_tensor(sc["length"]))
    Xh = api.mlp_features(sch, torch.as_tensor(sc["p_init"]), torch.as_tensor(sc["v_init"]), K, DT,
                          torch.as_tensor(Yh), 1)
    th_learned = torch.as_tensor(synth.plain_init(1000), dtype=torch.float32, device="cuda").contiguous()
    net.predict_params(Xh, th_learned)
    # the prediction beats the training-label mean (the best input-free guess)
    lab_h = M.labels(sc["theta_true"], synth.BOX_LO, synth.BOX_HI)
    pred_h = M.labels(th_learned.double().cpu().numpy(), synth.BOX_LO, synth.BOX_HI)
    prior = lab.double().mean(0).cpu().numpy()
    assert np.mean((pred_h - lab_h) ** 2) < np.mean((prior - lab_h) ** 2)

    def fit_rmse(theta0, n_iter):
        th0 = torch.as_tensor(theta0, dtype=torch.float32, device="cuda").contiguous()
        api.fit(th0, torch.as_tensor(sc["p_init"]), torch.as_tensor(sc["v_init"]), sch, K, DT,
                torch.as_tensor(Yh), 1, n_iter)
        Pf, _ = oracle.forward(sc["lane_off"], sc["length"], th0.double().cpu().numpy(), sc["p_init"],
                               sc["v_init"], K, DT, A_MIN)
        return float(np.sqrt(np.mean((Pf[1:K + 1] - clean) ** 2)))

    r_plain = fit_rmse(synth.plain_init(1000), 30)
    r_learned = fit_rmse(th_learned.double().cpu().numpy(), 30)
    assert r_learned < r_plain, (r_learned, r_plain)


def test_predict_params_large_chunks_match_one_pass(api):
    """More rows than one inference chunk (131,072): the chunked pass through
    the network's inference buffers equals one pass through the training
    buffers of a network sized for all rows (same kernels per row)."""
    B = 131072 + 1000
    w = synth.mlp_init(5)
    rng = np.random.default_rng(70)
    X = to_bf16_cuda(rng.normal(scale=0.7, size=(B, 80)))
    a, b = api.Mlp(max_batch=1024, weights=w), api.Mlp(max_batch=B, weights=w)
    ta = torch.zeros((6, B), device="cuda", dtype=torch.float32)
    tb = torch.zeros((6, B), device="cuda", dtype=torch.float32)
    a.predict_params(X, ta)
    b.predict_params(X, tb)
    torch.cuda.synchronize()
    assert torch.equal(ta, tb)
    assert a.status() == (0, 0) and b.status() == (0, 0)


def test_persistent_gemm_path_matches_oracle(api):
    """A batch large enough (>= 2 row tiles per SM) for the persistent
    weight-stationary kernel in every batch-sized product: forward outputs,
    loss and gradients against the FP64 oracle."""
    B = 2 * 152 * 128 + 77
    w = synth.mlp_init(6)
    X, T = random_batch(B, 80)
    Xc, Tc = to_bf16_cuda(X), torch.as_tensor(T, dtype=torch.float32, device="cuda")
    net = api.Mlp(max_batch=B, weights=w)
    wb = bf16_weights(w)
    S = net.forward(Xc).double().cpu().numpy()
    np.testing.assert_allclose(S, M.forward(wb, X)["s"], rtol=1e-2, atol=1e-3)
    loss, g = net.loss_grad(Xc, Tc)
    torch.cuda.synchronize()
    L_ref, g_ref = M.loss_grad(wb, X, synth.f32(T))
    assert abs(loss.item() - L_ref) <= 1e-2 * L_ref
    gd, rd = M.unpack(g.double().cpu().numpy()), M.unpack(g_ref)
    for name, _ in M.SHAPES:
        assert cosine(gd[name], rd[name]) >= 0.999, name
    assert net.status() == (0, 0)


def test_gelu_approximation_error_bound(api):
    """The kernels' GELU and its derivative (erf by Abramowitz & Stegun
    7.1.26, |error| <= 1.5e-7) against the FP64 closed forms."""
    from math import erf, exp, pi, sqrt
    from paper_2412_16750_gb300 import lib
    z = np.concatenate([np.linspace(-9, 9, 20001), np.random.default_rng(90).normal(scale=3, size=20000)])
    z = z.astype(np.float32)
    zt = torch.as_tensor(z, device="cuda")
    g = torch.empty_like(zt)
    dg = torch.empty_like(zt)
    assert lib.idm_mlp_gelu_eval(zt, g, dg) == lib.IDM_OK
    torch.cuda.synchronize()
    zd = z.astype(np.float64)
    cdf = np.array([0.5 * (1 + erf(x / sqrt(2))) for x in zd])
    pdf = np.exp(-0.5 * zd * zd) / sqrt(2 * pi)
    tol = 4e-7 * np.maximum(1.0, np.abs(zd))
    assert np.all(np.abs(g.double().cpu().numpy() - zd * cdf) <= tol)
    assert np.all(np.abs(dg.double().cpu().numpy() - (cdf + zd * pdf)) <= tol)


@pytest.mark.parametrize("B", [1000, 2 * 152 * 128 + 77])
def test_bounded_wait_gives_up_then_recovers(api, B):
    """A tensor-core wait limited to one poll cannot see its copies or MMAs
    finish: the kernel sets IDM_STATUS_TIMEOUT, drains what it issued, frees
    its tensor memory and returns (the host sees IDM_ERR_TIMEOUT).  With the
    default limit back, the same calls succeed and match the oracle, so the
    context is usable and the tensor memory was released.  B = 1000 runs the
    per-tile GEMM, the larger batch the persistent weight-stationary one;
    loss_grad adds the split-K weight-gradient GEMMs."""
    from paper_2412_16750_gb300 import lib
    w = synth.mlp_init(7)
    X, T = random_batch(B, 90)
    Xc, Tc = to_bf16_cuda(X), torch.as_tensor(T, dtype=torch.float32, device="cuda")
    net = api.Mlp(max_batch=B, weights=w)
    net.set_wait_limit(1)
    net.forward(Xc)
    rc, bits = net.status()
    assert rc == lib.IDM_ERR_TIMEOUT and bits & lib.IDM_STATUS_TIMEOUT
    net.clear_status()
    net.loss_grad(Xc, Tc)
    rc, bits = net.status()
    assert rc == lib.IDM_ERR_TIMEOUT and bits & lib.IDM_STATUS_TIMEOUT
    net.set_wait_limit(0)
    net.clear_status()
    assert net.status() == (0, 0)
    wb = bf16_weights(w)
    S = net.forward(Xc).double().cpu().numpy()
    np.testing.assert_allclose(S, M.forward(wb, X)["s"], rtol=1e-2, atol=1e-3)
    loss, g = net.loss_grad(Xc, Tc)
    torch.cuda.synchronize()
    L_ref, g_ref = M.loss_grad(wb, X, synth.f32(T))
    assert abs(loss.item() - L_ref) <= 1e-2 * L_ref
    gd, rd = M.unpack(g.double().cpu().numpy()), M.unpack(g_ref)
    for name, _ in M.SHAPES:
        assert cosine(gd[name], rd[name]) >= 0.999, name
    assert net.status() == (0, 0)
