"""Multi-GPU (multi-rank) fits: lanes are independent in the forward, the
adjoint and Adam (the leader of a vehicle is in its own lane, Sec. III-A, and
every parameter belongs to one vehicle), so a scene shards into contiguous
lane ranges and a batch of scenarios into contiguous scenario ranges, with
no exchange on the data path.  The one collective is the sum of the ranks'
FP64 loss histories (the scene's loss is the sum of its lanes' losses); the
timers are reduced with a max.

    fit_sharded        one scene, each rank fits its lane range (idm_fit on
                       its GPU, or idm_cpu_fit on its host cores)
    batch_fit_sharded  a batch of scenarios, each rank fits its scenario range
                       (idm_batch_fit)

Both take the whole problem as host arrays (what every rank can generate or
read); a rank copies only its own range to its device.
"""
import numpy as np


def lane_shards(lane_off, world, steps=None):
    """Contiguous lane ranges [(l0, l1)] per rank, balanced by vehicles x
    steps (steps: per-lane horizons, default all equal)."""
    lane_off = np.asarray(lane_off, dtype=np.int64)
    L = len(lane_off) - 1
    w = np.diff(lane_off).astype(np.float64)
    if steps is not None:
        w = w * np.asarray(steps, dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        l = int(np.searchsorted(cum, total * r / world, side="left"))
        l = min(max(l, cuts[-1]), L)
        cuts.append(l)
    cuts.append(L)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def scenario_shards(veh_counts, K, world):
    """Contiguous scenario ranges [(s0, s1)] per rank, balanced by the sum of
    vehicles x horizon of the scenarios."""
    off = np.concatenate([[0], np.cumsum(np.asarray(veh_counts, dtype=np.int64))])
    return lane_shards(off, world, steps=K)


def shard_arrays(lane_off, l0, l1):
    """Vehicle range and rebased lane CSR of the lanes [l0, l1)."""
    lane_off = np.asarray(lane_off, dtype=np.int64)
    a, e = int(lane_off[l0]), int(lane_off[l1])
    return a, e, (lane_off[l0:l1 + 1] - a).astype(np.int32)


def _world():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def all_reduce_scalar(x, op="sum", device=None):
    """float64 all-reduce of one scalar over the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t.item())


def _all_reduce_hist(hist, device=None):
    """Sum of the ranks' FP64 loss histories (numpy in, numpy out)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(hist, dtype=np.float64), device=device).clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def fit_sharded(lane_off, length, theta, p_init, v_init, K, dt, targets, obs_stride, n_iter, lr0=0.1, lr1=0.01,
                box_lo=(20.0, 0.1, 1.0, 0.5, 0.1), box_hi=(60.0, 5.0, 10.0, 10.0, 5.0), a_min=-10.0, backend="cuda",
                ctx=None, threads=0):
    """Fit one scene across the ranks of the default process group (or
    alone when there is none).

    lane_off [L+1], length [N], theta (6, N), p_init, v_init [N] and targets
    [K // obs_stride][N] are host arrays of the WHOLE scene (time-major
    targets).  Rank r fits the lanes lane_shards(lane_off, world)[r]:
    backend "cuda" with idm_fit on the current CUDA device, "cpu" with
    idm_cpu_fit on the host cores (`threads`, 0 = all).  The FP64 loss
    histories of the shards are summed across ranks.

    Returns (theta_shard float32 (6, e - a), (a, e) its vehicle range,
    loss_hist float64 (n_iter,) of the whole scene)."""
    rank, world = _world()
    l0, l1 = lane_shards(lane_off, world)[rank]
    a, e, lo = shard_arrays(lane_off, l0, l1)
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32)[:, a:e])
    tg = np.ascontiguousarray(np.asarray(targets, dtype=np.float32)[:, a:e])
    n_hist = max(n_iter, 0)
    if e == a:          # an empty shard contributes nothing, but joins the collective
        hist = np.zeros(n_hist)
        dev = None
    elif backend == "cpu":
        from . import cpu
        hist = cpu.idm_cpu_fit(th, np.asarray(p_init)[a:e], np.asarray(v_init)[a:e],
                               cpu.Scene(lo, np.asarray(length)[a:e]), K, dt, tg, obs_stride, n_iter, lr0, lr1,
                               box_lo, box_hi, a_min, threads)
        dev = None
    elif backend == "cuda":
        import torch
        from . import api
        cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device="cuda")
        scene = api.Scene.from_lane_off(cu(lo, torch.int32), cu(np.asarray(length)[a:e]))
        th_d = cu(th)
        h = api.fit(th_d, cu(np.asarray(p_init)[a:e]), cu(np.asarray(v_init)[a:e]), scene, K, dt, cu(tg), obs_stride,
                    n_iter, lr0, lr1, box_lo, box_hi, a_min, ctx=ctx)
        th = th_d.cpu().numpy()
        hist = h.cpu().numpy()
        dev = None
    else:
        raise ValueError("backend must be 'cuda' or 'cpu'")
    return th, (a, e), _all_reduce_hist(hist[:n_hist], dev)


def batch_fit_sharded(scen_lane_off, K, dt, obs_stride, lane_off, length, theta, p_init, v_init, targets, n_iter,
                      lr0=0.1, lr1=0.01, box_lo=(20.0, 0.1, 1.0, 0.5, 0.1), box_hi=(60.0, 5.0, 10.0, 10.0, 5.0),
                      a_min=-10.0, ctx=None):
    """Fit a batch of scenarios (the idm_batch_* layout) across the ranks:
    rank r takes the scenarios scenario_shards(...)[r], balanced by vehicles
    x horizon, and runs idm_batch_fit on them on the current CUDA device.

    Host arrays of the WHOLE batch: scen_lane_off [S+1], K, dt, obs_stride
    [S], lane_off [L+1], length / p_init / v_init [N], theta (6, N) and the
    flat concatenated per-scenario targets (scenario order, each [n_obs][n_veh]).
    Returns (theta_shard (6, e - a), (a, e) its vehicle range, (s0, s1) its
    scenarios, loss_hist float64 (n_iter,) summed over all scenarios)."""
    import torch
    from . import api
    rank, world = _world()
    scen_lane_off = np.asarray(scen_lane_off, dtype=np.int64)
    lane_off = np.asarray(lane_off, dtype=np.int64)
    K = np.asarray(K, dtype=np.int32)
    obs_stride = np.asarray(obs_stride, dtype=np.int32)
    veh_off = lane_off[scen_lane_off]
    nv = np.diff(veh_off)
    s0, s1 = scenario_shards(nv, K, world)[rank]
    a, e = int(veh_off[s0]), int(veh_off[s1])
    n_obs = (K // obs_stride).astype(np.int64)
    tgt_off = np.concatenate([[0], np.cumsum(n_obs * nv)])
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32)[:, a:e])
    if s1 == s0:
        return th, (a, e), (s0, s1), _all_reduce_hist(np.zeros(max(n_iter, 0)))
    L0, L1 = int(scen_lane_off[s0]), int(scen_lane_off[s1])
    b = api.Batch(scen_lane_off[s0:s1 + 1] - L0, K[s0:s1], np.asarray(dt, np.float32)[s0:s1], obs_stride[s0:s1],
                  lane_off[L0:L1 + 1] - a, np.asarray(length)[a:e], a_min)
    cu = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")
    th_d = cu(th)
    tg = cu(np.asarray(targets, dtype=np.float32)[tgt_off[s0]:tgt_off[s1]])
    hist, _ = api.batch_fit(th_d, cu(np.asarray(p_init)[a:e]), cu(np.asarray(v_init)[a:e]), b, tg, n_iter, lr0, lr1,
                            box_lo, box_hi, ctx=ctx)
    return th_d.cpu().numpy(), (a, e), (s0, s1), _all_reduce_hist(hist.cpu().numpy())


def weak_scaling_value(units_per_rank, world, ms_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)
