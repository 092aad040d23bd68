"""The product path of the multi-rank fit on the GPU: dist.fit_sharded and
dist.batch_fit_sharded on two gloo ranks, each fitting its share (lane range
or scenario range) with libidm on the one GPU of this machine (separate
processes and contexts; no kernel of one rank waits on the other, the only
exchange is the host-side FP64 loss-history sum).  Every rank's parameters
equal its slice of the unsharded fit bit for bit (lanes and scenarios never
interact); the summed loss history equals the unsharded one up to the order
of the FP64 sums."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2412_16750_gb300 import dist as idm_dist
from paper_2412_16750_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = float(np.float32(0.1))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scene_problem():
    sc = synth.make_scene([100, 40, 100, 7, 100, 100, 64, 100, 1, 100], np.random.default_rng(500))
    K = 120
    N = int(sc["lane_off"][-1])
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT)
    Y = synth.f32(P[1:] + np.random.default_rng(501).normal(0, 0.5, size=(K, N)))
    return sc, K, Y, synth.plain_init(N)


def _batch_problem():
    rng = np.random.default_rng(502)
    lanes = rng.integers(1, 6, 9)
    counts = [list(rng.integers(2, 60, n)) for n in lanes]
    K = rng.integers(30, 150, 9).astype(np.int32)
    stride = np.array([1, 2, 10, 1, 3, 1, 5, 1, 2], np.int32)
    flat = [c for cs in counts for c in cs]
    sc = synth.make_scene(flat, rng)
    scen_lane_off = np.concatenate([[0], np.cumsum(lanes)]).astype(np.int32)
    veh_off = sc["lane_off"][scen_lane_off]
    tg = []
    for q in range(9):
        a, e = int(veh_off[q]), int(veh_off[q + 1])
        lo = (sc["lane_off"][scen_lane_off[q]:scen_lane_off[q + 1] + 1] - a).astype(np.int32)
        P, _ = oracle.forward(lo, sc["length"][a:e], sc["theta_true"][:, a:e], sc["p_init"][a:e], sc["v_init"][a:e],
                              int(K[q]), DT)
        n = int(K[q]) // int(stride[q])
        tg.append((P[stride[q]::stride[q]][:n] + rng.normal(0, 0.5, size=(n, e - a))).ravel())
    return sc, scen_lane_off, K, stride, synth.f32(np.concatenate(tg)), synth.plain_init(int(sc["lane_off"][-1]))


def _rank(rank, world, port, out, kind):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    if kind == "scene":
        sc, K, Y, th0 = _scene_problem()
        th, (a, e), hist = idm_dist.fit_sharded(sc["lane_off"], sc["length"], th0, sc["p_init"], sc["v_init"], K, DT,
                                                Y, 1, 8, backend="cuda")
    else:
        sc, slo, K, stride, Y, th0 = _batch_problem()
        th, (a, e), _, hist = idm_dist.batch_fit_sharded(slo, K, np.full(len(K), DT, np.float32), stride,
                                                         sc["lane_off"], sc["length"], th0, sc["p_init"],
                                                         sc["v_init"], Y, 8)
    torch.cuda.synchronize()
    out.put((rank, a, e, th, hist))
    dist.barrier()
    dist.destroy_process_group()


def _spawn(kind, world=2):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, kind)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


def test_fit_sharded_cuda_backend():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16750_gb300 import api
    sc, K, Y, th0 = _scene_problem()
    cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device="cuda")
    th = cu(th0)
    h_full = api.fit(th, cu(sc["p_init"]), cu(sc["v_init"]),
                     api.Scene.from_lane_off(cu(sc["lane_off"], torch.int32), cu(sc["length"])), K, DT, cu(Y), 1, 8)
    th_full, h_full = th.cpu().numpy(), h_full.cpu().numpy()
    covered = np.zeros(th0.shape[1], dtype=bool)
    for rank, a, e, th_r, hist in _spawn("scene"):
        assert e > a
        np.testing.assert_array_equal(th_r, th_full[:, a:e])
        np.testing.assert_allclose(hist, h_full, rtol=1e-12)
        covered[a:e] = True
    assert covered.all()


def test_batch_fit_sharded_cuda_backend():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16750_gb300 import api
    sc, slo, K, stride, Y, th0 = _batch_problem()
    cu = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")
    b = api.Batch(slo, K, np.full(len(K), DT, np.float32), stride, sc["lane_off"], sc["length"])
    th = cu(th0)
    h_full, _ = api.batch_fit(th, cu(sc["p_init"]), cu(sc["v_init"]), b, cu(Y), 8)
    th_full, h_full = th.cpu().numpy(), h_full.cpu().numpy()
    covered = np.zeros(th0.shape[1], dtype=bool)
    for rank, a, e, th_r, hist in _spawn("batch"):
        assert e > a
        np.testing.assert_array_equal(th_r, th_full[:, a:e])
        np.testing.assert_allclose(hist, h_full, rtol=1e-12)
        covered[a:e] = True
    assert covered.all()
