"""Multi-rank path on CPU (gloo): lane and scenario sharding and the host-side
collectives.  The sharded loss equals the unsharded one and every rank's
gradients equal its slice of the full adjoint (FP64 oracle); the product
path dist.fit_sharded, driving libidm_cpu.so on every rank, reproduces the
unsharded fit of the same library."""
import os
import socket

import numpy as np
import pytest

from paper_2412_16750_gb300 import dist as idm_dist
from paper_2412_16750_gb300 import synth

torch = pytest.importorskip("torch")


def test_lane_shards_balanced_and_complete():
    lane_off = synth.lane_offsets([5, 100, 3, 40, 40, 7, 90, 1])
    for world in (1, 2, 3, 4, 8):
        sh = idm_dist.lane_shards(lane_off, world)
        assert sh[0][0] == 0 and sh[-1][1] == 8
        assert all(sh[r][1] == sh[r + 1][0] for r in range(world - 1))
    sh = idm_dist.lane_shards(synth.lane_offsets([100] * 20), 4)
    assert [b - a for a, b in sh] == [5, 5, 5, 5]
    assert idm_dist.weak_scaling_value(1e9, 4, 1000.0) == pytest.approx(4e9)


def test_lane_shards_balance_vehicle_steps():
    """Weights per lane (vehicles x horizon) move the cuts; scenario shards
    balance the sum of vehicles x horizon."""
    lane_off = synth.lane_offsets([10, 10, 10, 10])
    assert idm_dist.lane_shards(lane_off, 2) == [(0, 2), (2, 4)]
    assert idm_dist.lane_shards(lane_off, 2, steps=[300, 100, 100, 100]) == [(0, 1), (1, 4)]
    sh = idm_dist.scenario_shards([100, 50, 50, 100], [100, 200, 200, 100], 2)
    assert sh == [(0, 2), (2, 4)]
    rng = np.random.default_rng(5)
    nv, K = rng.integers(2, 200, 500), rng.integers(50, 500, 500)
    for world in (2, 3, 8):
        sh = idm_dist.scenario_shards(nv, K, world)
        w = [int(np.sum(nv[a:b] * K[a:b])) for a, b in sh]
        assert sum(w) == int(np.sum(nv * K))
        assert max(w) - min(w) <= 2 * int(np.max(nv * K))    # within two scenarios of even


def test_lane_shards_more_ranks_than_lanes():
    lane_off = synth.lane_offsets([4, 9, 2])
    sh = idm_dist.lane_shards(lane_off, 8)
    assert len(sh) == 8 and sh[0][0] == 0 and sh[-1][1] == 3
    assert all(sh[r][1] == sh[r + 1][0] and sh[r][0] <= sh[r][1] for r in range(7))
    assert sum(b - a for a, b in sh) == 3
    for a_l, b_l in sh:   # an empty shard has an empty vehicle range and a one-entry CSR
        a, e, lo = idm_dist.shard_arrays(lane_off, a_l, b_l)
        assert e - a == int(lane_off[b_l] - lane_off[a_l]) and len(lo) == b_l - a_l + 1 and lo[0] == 0


def test_sharded_fit_equals_unsharded():
    """Lanes never interact and Adam is per vehicle, so fitting each rank's
    lanes alone (FP64 oracle) reproduces the unsharded fit, and the per-rank
    loss histories sum to the unsharded history."""
    import oracle
    sc = synth.make_scene([7, 12, 3, 9, 15, 4, 1], np.random.default_rng(42))
    K, dt, n_iter = 20, float(np.float32(0.1)), 4
    N = int(sc["lane_off"][-1])
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, dt)
    Y = P[1:] + np.random.default_rng(43).normal(0, 0.5, size=(K, N))
    th0 = synth.plain_init(N)
    th_full, h_full = oracle.fit(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K, dt, Y, 1, n_iter,
                                 0.1, 0.01, synth.BOX_LO, synth.BOX_HI)
    for world in (2, 3):
        h_sum = np.zeros(n_iter)
        for l0, l1 in idm_dist.lane_shards(sc["lane_off"], world):
            a, e, lo = idm_dist.shard_arrays(sc["lane_off"], l0, l1)
            th, h = oracle.fit(lo, sc["length"][a:e], th0[:, a:e], sc["p_init"][a:e], sc["v_init"][a:e], K, dt,
                               Y[:, a:e], 1, n_iter, 0.1, 0.01, synth.BOX_LO, synth.BOX_HI)
            np.testing.assert_allclose(th, th_full[:, a:e], rtol=1e-12, atol=1e-13)
            h_sum += h
        np.testing.assert_allclose(h_sum, h_full, rtol=1e-12)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = synth.make_scene([7, 12, 3, 9, 15, 4], np.random.default_rng(40))
    K, dt = 25, float(np.float32(0.1))
    N = int(sc["lane_off"][-1])
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, dt)
    Y = P[1:] + np.random.default_rng(41).normal(0, 0.5, size=(K, N))
    theta = synth.plain_init(N)
    l0, l1 = idm_dist.lane_shards(sc["lane_off"], world)[rank]
    a, e, lo = idm_dist.shard_arrays(sc["lane_off"], l0, l1)
    Ps, Vs = oracle.forward(lo, sc["length"][a:e], theta[:, a:e], sc["p_init"][a:e], sc["v_init"][a:e], K, dt)
    L, gP = oracle.mse_seed(Ps, Y[:, a:e], 1)
    g, _, _ = oracle.adjoint(lo, sc["length"][a:e], theta[:, a:e], K, dt, Ps, Vs, gP)
    total = idm_dist.all_reduce_scalar(L, "sum")
    slowest = idm_dist.all_reduce_scalar(float(rank + 1), "max")
    out.put((rank, a, e, L, total, slowest, g))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_loss_and_gradients_match_unsharded():
    import multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = synth.make_scene([7, 12, 3, 9, 15, 4], np.random.default_rng(40))
    K, dt = 25, float(np.float32(0.1))
    N = int(sc["lane_off"][-1])
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, dt)
    Y = P[1:] + np.random.default_rng(41).normal(0, 0.5, size=(K, N))
    theta = synth.plain_init(N)
    Pf, Vf = oracle.forward(sc["lane_off"], sc["length"], theta, sc["p_init"], sc["v_init"], K, dt)
    Lf, gPf = oracle.mse_seed(Pf, Y, 1)
    gf, _, _ = oracle.adjoint(sc["lane_off"], sc["length"], theta, K, dt, Pf, Vf, gPf)
    covered = np.zeros(N, dtype=bool)
    for rank, a, e, L, total, slowest, g in res:
        assert total == pytest.approx(Lf, rel=1e-12)
        assert slowest == 2.0
        np.testing.assert_allclose(g, gf[:, a:e], rtol=1e-12, atol=1e-15)
        covered[a:e] = True
    assert covered.all()


def _fit_problem(seed=44):
    import oracle
    sc = synth.make_scene([7, 12, 3, 9, 15, 4, 1, 20, 6], np.random.default_rng(seed))
    K, dt = 30, float(np.float32(0.1))
    N = int(sc["lane_off"][-1])
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, dt)
    Y = synth.f32(P[1:] + np.random.default_rng(seed + 1).normal(0, 0.5, size=(K, N)))
    return sc, K, dt, Y, synth.plain_init(N)


def _rank_fit(rank, world, port, out):
    import torch.distributed as dist
    from paper_2412_16750_gb300 import build
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    build.build_cpu()
    sc, K, dt, Y, th0 = _fit_problem()
    th, (a, e), hist = idm_dist.fit_sharded(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K, dt, Y,
                                            1, 6, backend="cpu", threads=2)
    out.put((rank, a, e, th, hist))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_fit_sharded_product_path(world):
    """dist.fit_sharded on gloo ranks, each fitting its lane range with the
    CPU backend (libidm_cpu.so): every rank's parameters equal its slice of
    the unsharded fit bit for bit (lanes never interact), and the all-reduced
    loss history equals the unsharded one up to the order of the FP64 sum."""
    import multiprocessing as mp
    from paper_2412_16750_gb300 import build, cpu
    build.build_cpu()
    sc, K, dt, Y, th0 = _fit_problem()
    th_full = th0.astype(np.float32).copy()
    h_full = cpu.idm_cpu_fit(th_full, sc["p_init"], sc["v_init"], cpu.Scene(sc["lane_off"], sc["length"]), K, dt, Y,
                             1, 6, threads=2)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_fit, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    covered = np.zeros(th0.shape[1], dtype=bool)
    for rank, a, e, th, hist in res:
        np.testing.assert_array_equal(th, th_full[:, a:e])
        np.testing.assert_allclose(hist, h_full, rtol=1e-12)
        covered[a:e] = True
    assert covered.all()
