"""Multi-GPU helpers: lanes are independent in the forward, the adjoint and
Adam, so a scene shards into contiguous lane ranges with no data-path
collective.  The only collectives are host-side bookkeeping: a max of the
per-rank timers and a sum of the per-rank losses (both float64 scalars).
"""
import numpy as np


def lane_shards(lane_off, world):
    """Contiguous lane ranges [(l0, l1)] per rank, balanced by vehicle count."""
    lane_off = np.asarray(lane_off, dtype=np.int64)
    L = len(lane_off) - 1
    N = int(lane_off[-1])
    cuts = [0]
    for r in range(1, world):
        target = N * r / world
        l = int(np.searchsorted(lane_off, target, side="left"))
        l = min(max(l, cuts[-1]), L)
        cuts.append(l)
    cuts.append(L)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard_arrays(lane_off, l0, l1):
    """Vehicle range and rebased lane CSR of the lanes [l0, l1)."""
    lane_off = np.asarray(lane_off, dtype=np.int64)
    a, e = int(lane_off[l0]), int(lane_off[l1])
    return a, e, (lane_off[l0:l1 + 1] - a).astype(np.int32)


def all_reduce_scalar(x, op="sum", device=None):
    """float64 all-reduce of one scalar over the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank, world, ms_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)
