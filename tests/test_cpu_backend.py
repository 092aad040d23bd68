"""The multi-threaded CPU backend (include/idm_cpu.h) against the FP64
oracle, on the CPU: the same tolerances as the CUDA path (positions 1e-3 m
over 100 steps; per-parameter relative gradient error 1e-4, every element
within 1e-3 of the largest), results independent of the thread count."""
import numpy as np
import pytest

import oracle
from paper_2412_16750_gb300 import synth

DT = float(np.float32(0.1))
A_MIN = -10.0


@pytest.fixture(scope="module")
def cpu():
    from paper_2412_16750_gb300 import build, cpu as _cpu
    build.build_cpu()
    return _cpu


def scene(cpu, counts, seed):
    sc = synth.make_scene(counts, np.random.default_rng(seed))
    return sc, cpu.Scene(sc["lane_off"], sc["length"])


def noisy(sc, K, s, seed):
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    rng = np.random.default_rng(seed)
    n = K // s
    return synth.f32(P[s::s][:n] + rng.normal(0, 0.5, size=(n, P.shape[1])))


def grad_close(g, ref, rtol=1e-4, elem=1e-3):
    for q in range(ref.shape[0]):
        nr = np.linalg.norm(ref[q])
        if nr == 0:
            assert np.max(np.abs(g[q])) == 0.0
            continue
        assert np.linalg.norm(g[q] - ref[q]) / nr <= rtol, q
        assert np.max(np.abs(g[q] - ref[q])) <= elem * np.max(np.abs(ref[q])), q


COUNTS = [0, 1, 2, 3, 17, 64, 100, 5]


def test_forward_parity(cpu):
    sc, s = scene(cpu, COUNTS, 1)
    th = synth.plain_init(len(sc["length"]))
    th[:, ::3] = sc["theta_true"][:, ::3]
    th[5, ::7] = 3.0
    traj, vtraj = cpu.idm_cpu_forward(th, sc["p_init"], sc["v_init"], s, 100, DT, A_MIN, want_speed=True)
    P, V = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], 100, DT, A_MIN)
    np.testing.assert_allclose(traj, P, rtol=0, atol=1e-3)
    np.testing.assert_allclose(vtraj, V, rtol=0, atol=1e-4)


@pytest.mark.parametrize("stride", [1, 7])
def test_loss_grad_parity(cpu, stride):
    sc, s = scene(cpu, COUNTS, 2)
    K = 100
    Y = noisy(sc, K, stride, 3)
    th = synth.plain_init(len(sc["length"]))
    th[:, ::2] = sc["theta_true"][:, ::2]
    L, g, gp, gv = cpu.idm_cpu_loss_grad(th, sc["p_init"], sc["v_init"], s, K, DT, Y, stride, A_MIN)
    P, V = oracle.forward(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, DT, A_MIN)
    Lr, gP = oracle.mse_seed(P, Y, stride)
    gr, gpr, gvr = oracle.adjoint(sc["lane_off"], sc["length"], th, K, DT, P, V, gP, None, A_MIN)
    assert abs(L - Lr) <= 1e-5 * Lr
    grad_close(g, gr)
    grad_close(gp[None], gpr[None])
    grad_close(gv[None], gvr[None])


def test_thread_count_invariance(cpu):
    sc, s = scene(cpu, [30] * 40 + [7, 1, 90], 4)
    K = 60
    Y = noisy(sc, K, 2, 5)
    th = synth.plain_init(len(sc["length"]))
    a = cpu.idm_cpu_loss_grad(th, sc["p_init"], sc["v_init"], s, K, DT, Y, 2, A_MIN, threads=1)
    b = cpu.idm_cpu_loss_grad(th, sc["p_init"], sc["v_init"], s, K, DT, Y, 2, A_MIN, threads=4)
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)


def test_fit_parity(cpu):
    sc, s = scene(cpu, [50] * 6 + [13], 6)
    K, stride, n_iter = 80, 2, 5
    Y = noisy(sc, K, stride, 7)
    th0 = synth.plain_init(len(sc["length"]))
    th_ref, hist_ref = oracle.fit(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K, DT, Y, stride,
                                  n_iter, 0.1, 0.01, synth.BOX_LO, synth.BOX_HI, A_MIN)
    th = th0.astype(np.float32).copy()
    hist = cpu.idm_cpu_fit(th, sc["p_init"], sc["v_init"], s, K, DT, Y, stride, n_iter, 0.1, 0.01, synth.BOX_LO,
                           synth.BOX_HI, A_MIN)
    np.testing.assert_allclose(hist, hist_ref, rtol=1e-5)
    np.testing.assert_allclose(th, th_ref, rtol=1e-4, atol=1e-5)


def test_argument_errors(cpu):
    sc, s = scene(cpu, [3, 4], 8)
    th = synth.plain_init(7)
    bad = cpu.Scene(np.array([0, 3, 2], np.int32), sc["length"])
    with pytest.raises(cpu.CpuError):
        cpu.idm_cpu_forward(th, sc["p_init"], sc["v_init"], bad, 10, DT)
    with pytest.raises(cpu.CpuError):
        cpu.idm_cpu_forward(th, sc["p_init"], sc["v_init"], s, 0, DT)
    with pytest.raises(cpu.CpuError):
        cpu.idm_cpu_loss_grad(th, sc["p_init"], sc["v_init"], s, 10, DT, np.zeros((10, 7)), 0)


def test_braking_to_rest_delta_gradient(cpu):
    # a creeping follower a few centimetres behind a stopped leader: its next
    # speed rounds below 0; the delta gradient must stay finite (r -> 0+ limit)
    rng = np.random.default_rng(81)
    p, v = [], []
    for _ in range(20):
        g1 = rng.uniform(0.02, 0.5)
        p += [0.0, -(5.0 + g1)]
        v += [0.0, rng.uniform(0.05, 0.9)]
    lane_off = synth.lane_offsets([2] * 20)
    length = np.full(40, 5.0)
    th = synth.plain_init(40)
    K = 30
    P, V = oracle.forward(lane_off, length, th, p, v, K, DT, A_MIN)
    Y = synth.f32(P[1:] + np.random.default_rng(82).normal(0, 0.5, size=(K, 40)))
    s = cpu.Scene(lane_off, length)
    L, g, gp, gv = cpu.idm_cpu_loss_grad(th, synth.f32(p), synth.f32(v), s, K, DT, Y, 1, A_MIN)
    assert np.isfinite(g).all()
    P, V = oracle.forward(lane_off, length, th, synth.f32(p), synth.f32(v), K, DT, A_MIN)
    Lr, gP = oracle.mse_seed(P, Y, 1)
    gr, _, _ = oracle.adjoint(lane_off, length, th, K, DT, P, V, gP, None, A_MIN)
    assert abs(L - Lr) <= 1e-5 * Lr
    grad_close(g, gr)
