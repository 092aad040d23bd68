"""Kernel-shape autotuner for the simulation kernels.

A shape is (vpt, warps_per_segment, ckpt_interval, warps_per_block) as taken
by idm_set_tuning: vehicles per thread and warps per lane segment fix the
segment capacity 32 * vpt * warps (lanes are packed into segments of that
size), the checkpoint interval sets the adjoint's recompute length and
shared-memory tape, and warps per block the persistent grid.  The best shape
depends on the lane-length mix, the horizon and the GPU, so it is measured:
the caller supplies one run of its workload (a loss + gradient or a fit
iteration), the tuner times it for candidate shapes with CUDA events and
keeps the fastest.  Results are cached in a JSON file keyed by the GPU name
and a bucketed problem signature, so a later process with a similar problem
reuses them without timing.

Search: (vpt, warps) over all pairs whose capacity holds the longest lane,
at checkpoint interval 8 and 8 warps per block; then the checkpoint interval
for the best pair; then the warps per block.  Shapes the library rejects
(shared memory, capacity) are skipped.
"""
import json
import math
import os
import threading

_lock = threading.Lock()

VPT = (2, 4, 8)
WARPS = (1, 2, 4, 8)
CKPT = (4, 8, 16, 32)
WPB = (4, 8, 16)


def cache_path():
    p = os.environ.get("IDM_TUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "paper_2412_16750_gb300", "tune.json")


def _bucket(x):
    """Power-of-two bucket of a positive size."""
    return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))


def signature(max_lane, n_vehicles, mean_K, obs_stride=1, kind="loss_grad"):
    """Bucketed description of a problem: shapes tuned for one signature
    serve every problem with the same buckets."""
    return "%s|lane<=%d|N~%d|K~%d|s=%d" % (kind, _bucket(max_lane), _bucket(n_vehicles), _bucket(mean_K),
                                          int(obs_stride))


def load_cache(path=None):
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(device_name, sig, shape, ms, path=None):
    """Record shape (and its time) for (device, signature); atomic rewrite."""
    path = path or cache_path()
    with _lock:
        d = load_cache(path)
        d.setdefault(device_name, {})[sig] = {"shape": list(shape), "ms": ms}
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = "%s.tmp%d" % (path, os.getpid())
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def lookup(device_name, sig, path=None):
    e = load_cache(path).get(device_name, {}).get(sig)
    return tuple(e["shape"]) if e else None


def candidates_pairs(max_lane):
    return [(v, g) for v in VPT for g in WARPS if 32 * v * g >= max(1, max_lane)]


def search(time_shape, max_lane):
    """Staged search.  time_shape(shape) returns milliseconds, or None when
    the shape is rejected.  Returns (best shape, ms, every timing)."""
    timings = {}

    def t(shape):
        if shape not in timings:
            timings[shape] = time_shape(shape)
        return timings[shape]

    best, best_ms = None, float("inf")
    for v, g in candidates_pairs(max_lane):
        ms = t((v, g, 8, 8))
        if ms is not None and ms < best_ms:
            best, best_ms = (v, g, 8, 8), ms
    if best is None:
        raise RuntimeError("no kernel shape accepted for max_lane %d" % max_lane)
    for c in CKPT:
        s = (best[0], best[1], c, best[3])
        ms = t(s)
        if ms is not None and ms < best_ms:
            best, best_ms = s, ms
    for w in WPB:
        if w % best[1]:
            continue
        s = (best[0], best[1], best[2], w)
        ms = t(s)
        if ms is not None and ms < best_ms:
            best, best_ms = s, ms
    return best, best_ms, timings


def cuda_timer(run, ctx, repeats=3):
    """time_shape for search(): applies the shape to ctx (api.Context), runs
    the workload once to warm up, then times `repeats` runs with CUDA events
    and returns the median in milliseconds (None if the library rejects the
    shape)."""
    import torch

    from . import lib

    def time_shape(shape):
        try:
            ctx.set_tuning(*shape)
            run(ctx)
            torch.cuda.synchronize()
        except lib.IdmError:
            torch.cuda.synchronize()
            return None
        ts = []
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            run(ctx)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[len(ts) // 2]

    return time_shape


def tuned(ctx, run, max_lane, sig, repeats=3, path=None, retune=False):
    """Apply the cached shape for sig to ctx, or search, cache and apply the
    best one.  Returns (shape, "cache" or "tuned", timings)."""
    import torch
    dev = torch.cuda.get_device_name()
    if not retune:
        shape = lookup(dev, sig, path)
        if shape is not None:
            ctx.set_tuning(*shape)
            return shape, "cache", {}
    best, ms, timings = search(cuda_timer(run, ctx, repeats), max_lane)
    store(dev, sig, best, ms, path)
    ctx.set_tuning(*best)
    return best, "tuned", timings
