"""The allocation-free entry point idm_loss_grad_noalloc.

Some callers cannot allocate device memory (a custom allocator owns it, a
fixed budget is checked up front, or the call sits where cudaMalloc is not
allowed).  idm_loss_grad_noalloc serves them from the library's static
scratch array.  This file is collected last so that a failure here leaves
every other test already run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2412_16750_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = float(np.float32(0.1))


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16750_gb300 import api, lib
    return api, lib


def cuda(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def test_noalloc_matches_loss_grad_twice(mods):
    api, lib = mods
    sc = synth.config0()
    rng = np.random.default_rng(300)
    N, K = 1000, sc["K"]
    Y = cuda(synth.f32(sc["p_init"][None, :] + np.arange(1, K + 1)[:, None] * DT * sc["v_init"][None, :]
                       + rng.normal(0, 0.5, size=(K, N))))
    theta = cuda(synth.plain_init(N))
    p0, v0 = cuda(sc["p_init"]), cuda(sc["v_init"])
    scene = api.Scene.from_lane_off(cuda(sc["lane_off"], torch.int32), cuda(sc["length"]))
    ctx = api.Context(ckpt_interval=8)
    loss_ref, g_ref, gp_ref, gv_ref = api.loss_grad(theta, p0, v0, scene, K, DT, Y, 1, ctx=ctx)
    torch.cuda.synchronize()
    g_ref = g_ref.double().cpu().numpy()
    for call in range(2):
        loss = torch.full((), -1.0, device="cuda", dtype=torch.float64)
        g = torch.full((6, N), float("nan"), device="cuda")
        gp = torch.full((N,), float("nan"), device="cuda")
        gv = torch.full((N,), float("nan"), device="cuda")
        status = torch.full((1,), 12345, device="cuda", dtype=torch.int32)
        rc = lib.idm_loss_grad_noalloc(scene.c(), lib.make_params(theta), p0, v0, lib.make_sim(K, DT), Y, 1, loss,
                                       lib.make_params(g), gp, gv, status, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert rc == lib.IDM_OK, call
        assert int(status.item()) == 0
        assert loss.item() == pytest.approx(loss_ref.item(), rel=1e-5)
        gn = g.double().cpu().numpy()
        for q in range(6):
            nr = np.linalg.norm(g_ref[q])
            assert np.linalg.norm(gn[q] - g_ref[q]) <= 1e-4 * nr + 1e-30, (call, q)
        np.testing.assert_allclose(gp.double().cpu().numpy(), gp_ref.double().cpu().numpy(), rtol=1e-4,
                                   atol=1e-4 * float(gp_ref.abs().max()))
        np.testing.assert_allclose(gv.double().cpu().numpy(), gv_ref.double().cpu().numpy(), rtol=1e-4,
                                   atol=1e-4 * float(gv_ref.abs().max()))


def test_noalloc_rejects_oversized_problem(mods):
    api, lib = mods
    sc = synth.make_scene([100] * 200, np.random.default_rng(301))  # 20,000 vehicles
    N, K = 20000, 1000  # 20,000 x 125 checkpoints > the static scratch
    scene = api.Scene.from_lane_off(cuda(sc["lane_off"], torch.int32), cuda(sc["length"]))
    theta = cuda(synth.plain_init(N))
    p0, v0 = cuda(sc["p_init"]), cuda(sc["v_init"])
    Y = torch.zeros((K, N), device="cuda")
    rc = lib.idm_loss_grad_noalloc(scene.c(), lib.make_params(theta), p0, v0, lib.make_sim(K, DT), Y, 1)
    assert rc == lib.IDM_ERR_WORKSPACE
