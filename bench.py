#!/usr/bin/env python
"""Benchmark of the differentiable IDM fit at paper scale on GB300.

Workload (one "step" = one pass of the whole hot path over one batch):
  20,000 lanes x 100 vehicles (2,000,000 vehicles), 1,000 Euler steps of
  dt = 0.1 s, targets = the true trajectory + N(0, 0.5^2) m noise at every
  step.  The batch arrives unsorted; a step runs
    layout   idm_layout (sort by lane / position) + idm_gather of the
             per-vehicle arrays + idm_gather_rows of the targets,
    fit      idm_fit: --iters iterations of {fused forward + squared-error
             loss + checkpoints, adjoint with checkpoint recompute + fused
             Adam/projection}, from the paper's zero-knowledge initial guess.
  The metric counts forward+backward vehicle-steps: iters x N x K per step.

Lines printed (rank 0, one JSON line):
  value     device throughput, inputs resident in HBM before the timed region;
  e2e       the same steps with every input copied host->device (pinned) and
            the fitted parameters + loss history copied back, inside the timer;
  roofline  the adjoint kernel (the dominant one), timed with CUDA events
            recorded inside the fit graph on its stream;
  cpu_baseline  the FP64 oracle on a bounded sample on every host core (one
            process per core), plus the single-core figure.

--impl reference times the FP64 CPU oracle (the only reference available:
the paper ships no code) on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank fits its own 2M-vehicle batch (lanes are
independent, no data-path collective): weak scaling.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd vehicle-steps/s at 2M vehicles; time-to-fit 0.5 m RMSE, learned vs plain"
UNIT = "vehicle-steps/s"
DT = float(np.float32(0.1))
A_MIN = -10.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--lanes", type=int, default=20000)
    p.add_argument("--per-lane", type=int, default=100)
    p.add_argument("--K", type=int, default=1000)
    p.add_argument("--iters", type=int, default=100, help="Adam iterations per step")
    p.add_argument("--e2e-steps", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--vpt", type=int, default=4)
    p.add_argument("--G", type=int, default=4, help="warps per segment")
    p.add_argument("--ckpt", type=int, default=50, help="checkpoint interval of the timed fit (the stated 50)")
    p.add_argument("--tuned-ckpt", type=int, default=8,
                   help="also time the step at this interval (0 = skip); reported as tuned_variant")
    p.add_argument("--tuned-steps", type=int, default=3)
    p.add_argument("--wpb", type=int, default=8)
    # learned-versus-plain initial guess (time to fit 0.5 m RMSE)
    p.add_argument("--no-init-experiment", action="store_true")
    p.add_argument("--init-only", action="store_true", help="run only the initializer experiment")
    p.add_argument("--init-train-lanes", type=int, default=100000, help="x 100 vehicles = training samples")
    p.add_argument("--mlp-batch", type=int, default=8192)
    p.add_argument("--mlp-epochs", type=int, default=2)
    p.add_argument("--fit-iters", type=int, default=500)
    p.add_argument("--rmse-target", type=float, default=0.5)
    # batched uneven scenarios (one graph-captured launch per fit iteration)
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batched-only", action="store_true", help="run only the batched-scenario measurement")
    p.add_argument("--batch-scen", type=int, default=4096)
    p.add_argument("--batch-iters", type=int, default=20)
    # long horizon: fit on the first 2,000 of 3,000 steps, predict the rest
    p.add_argument("--no-recon", action="store_true")
    p.add_argument("--no-crossover", action="store_true")
    p.add_argument("--no-pred", action="store_true")
    p.add_argument("--pred-only", action="store_true", help="run only the lane-geometry prediction measurement")
    p.add_argument("--pred-scen", type=int, default=10000)
    p.add_argument("--pred-iters", type=int, default=500)
    p.add_argument("--crossover-only", action="store_true", help="run only the CPU-backend / GPU crossover")
    p.add_argument("--recon-only", action="store_true", help="run only the filtering/reconstruction measurement")
    p.add_argument("--recon-iters", type=int, default=500)
    p.add_argument("--no-long-horizon", action="store_true")
    p.add_argument("--long-only", action="store_true", help="run only the initializer + long-horizon measurement")
    p.add_argument("--long-lanes", type=int, default=20000)
    p.add_argument("--long-iters", type=int, default=50)
    return p.parse_args()


def workload_name(a):
    return ("%d lanes x %d vehicles (%.1fM) per GPU, %d steps, dt 0.1 s, checkpoints every %d steps; per step: "
            "layout + %d-iteration Adam fit" % (a.lanes, a.per_lane, a.lanes * a.per_lane / 1e6, a.K, a.ckpt,
                                                a.iters))


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_sample(n_lanes=10, per_lane=100, K=1000, iters=3, seed=0):
    """Time the FP64 oracle fit (forward + loss + adjoint + Adam) on a bounded
    sample of the workload.  Returns (vehicle-steps/s, seconds, description)."""
    import oracle
    from paper_2412_16750_gb300 import synth
    sc = synth.make_scene([per_lane] * n_lanes, synth.rng_for(1, seed))
    P, _ = oracle.forward(sc["lane_off"], sc["length"], sc["theta_true"], sc["p_init"], sc["v_init"], K, DT, A_MIN)
    Y = synth.f32(P[1:] + synth.rng_for(1, seed + 1).normal(0, 0.5, size=P[1:].shape))
    th = synth.plain_init(n_lanes * per_lane)
    t0 = time.perf_counter()
    oracle.fit(sc["lane_off"], sc["length"], th, sc["p_init"], sc["v_init"], K, DT, Y, 1, iters, 0.1, 0.01,
               synth.BOX_LO, synth.BOX_HI, A_MIN)
    dt = time.perf_counter() - t0
    units = iters * n_lanes * per_lane * K
    desc = "%d lanes x %d vehicles x %d steps, %d fit iterations, FP64 single thread" % (n_lanes, per_lane, K, iters)
    return units / dt, dt, desc


def _oracle_task(args):
    seed, iters = args
    v, secs, _ = oracle_sample(iters=iters, seed=seed)
    return v * secs


def oracle_all_cores(iters=10):
    """The same oracle sample on every host core at once (one process per
    core, started with spawn; samples differ by seed).  Returns
    (vehicle-steps/s over the wall time of the parallel run, seconds, cores)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_task, [(1000 + s, 1) for s in range(cores)], chunksize=1)  # warm: imports, library
        t0 = time.perf_counter()
        units = pool.map(_oracle_task, [(2000 + s, iters) for s in range(cores)], chunksize=1)
        wall = time.perf_counter() - t0
    return sum(units) / wall, wall, cores


def run_reference(a, rank):
    if rank != 0:
        return 0
    for _ in range(max(1, min(a.warmup, 1))):
        oracle_sample(iters=1)
    times, vals = [], []
    desc = ""
    for _ in range(a.steps):
        v, dt, desc = oracle_sample(iters=1)
        vals.append(v)
        times.append(dt)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_ginst(sm_mhz, n_sm):
    """FP32-pipe instruction issue peak: n_SM x 128 lanes x clock (Ginstr/s)."""
    return n_sm * 128 * sm_mhz * 1e6 / 1e9


# Algorithmic work per vehicle-step of the adjoint launch, counted from the
# method's formulas: FP32 lane operations of the recompute of the forward
# step (30) and of the reverse step with the gradient accumulation (80), and
# the special-function operations (exp2 / log2 / reciprocal: 5 in the
# recompute, 3 in the reverse step) on their own pipe.
ADJ_FP32_PER_VS = 110.0
ADJ_SFU_PER_VS = 8.0
SFU_PER_SM_CLK = 16


# Sources of the adjoint kernel: a committed ncu summary records their hash.
ADJOINT_SOURCES = ("idm_adjoint.cuh", "idm_sim_common.cuh", "idm_device.cuh")


def adjoint_traffic(n_vehicles, K, ckpt):
    """DRAM bytes of one adjoint launch (N K a + N b) from the committed ncu
    summary taken at this checkpoint interval (profiles/adjoint_kernel_*.md
    with a matching `ckpt_interval:` line), or None if there is none or it
    was taken on a different kernel source."""
    import glob
    import hashlib
    src = b""
    for name in ADJOINT_SOURCES:
        src += open(os.path.join(ROOT, "paper_2412_16750_gb300", "csrc", name), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "adjoint_kernel_*.md"))):
        got = {}
        for line in open(path):
            for key in ("kernel_source_sha256_16", "ckpt_interval", "dram_bytes_per_vehicle_step",
                        "dram_bytes_per_vehicle"):
                if line.startswith(key + ":"):
                    got[key] = line.split(":", 1)[1].strip()
        if got.get("kernel_source_sha256_16") != sha or got.get("ckpt_interval") != str(ckpt):
            continue
        if "dram_bytes_per_vehicle_step" not in got:
            continue
        return n_vehicles * K * float(got["dram_bytes_per_vehicle_step"]) + \
            n_vehicles * float(got.get("dram_bytes_per_vehicle", 0.0))
    return None


def adjoint_roofline(N, K, ckpt, bwd_avg_ms, n_sm, peaks, peak_kind):
    """Roofline object of the adjoint launch: bound by the FP32 pipe
    (algorithmic FP32 lane operations / launch time against 128 FP32 lanes
    per SM at the maximum SM clock), with the special-function pipe and HBM
    beside it."""
    units = N * K
    t = bwd_avg_ms * 1e-3
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    achieved = ADJ_FP32_PER_VS * units / t / 1e9
    peak = alu_peak_ginst(sm_mhz, n_sm)
    sfu_achieved = ADJ_SFU_PER_VS * units / t / 1e9
    sfu_peak = n_sm * SFU_PER_SM_CLK * sm_mhz * 1e6 / 1e9
    return {
        "kernel": "backward_kernel (adjoint with checkpoint recompute + fused Adam)",
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "G FP32 lane-ops/s",
        "frac": achieved / peak,
        "traffic": adjoint_traffic(N, K, ckpt),
        "peak_source": "nominal: %d SMs x 128 FP32 lanes x %.0f MHz (the maximum SM clock of MEASURED_PEAKS.json, "
                       "%s; that file has no FP32 figure)" % (n_sm, sm_mhz, peak_kind),
        "ops_per_vehicle_step": ADJ_FP32_PER_VS,
        "avg_launch_ms": bwd_avg_ms,
        "ckpt_interval": ckpt,
        "sfu": {"ops_per_vehicle_step": ADJ_SFU_PER_VS, "achieved": sfu_achieved, "peak": sfu_peak,
                "frac": sfu_achieved / sfu_peak, "unit": "G special-function ops/s",
                "peak_source": "nominal: %d SMs x %d per clock x %.0f MHz" % (n_sm, SFU_PER_SM_CLK, sm_mhz)},
        "hbm_achieved_gbs": (4.0 + 16.0 / ckpt) * units / t / 1e9,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }


def run_e2e(a, e2e_steps, step, barrier, max_over_ranks, stream, dev, u_lane, u_p, u_v, u_len, u_th, u_Y, s_th,
            hist, h, lib):
    """Time e2e_steps steps whose inputs start in pinned host memory and whose
    fitted parameters and loss history end in pinned host memory.  The inputs
    of step i + 1 are copied on a second stream into the other of two device
    buffers while step i computes (a copy waits until the step two back has
    released its buffer; a step waits for its own copy); every copy is inside
    the timed region."""
    import torch
    h_lane = u_lane.cpu().pin_memory()
    h_p, h_v, h_len = u_p.cpu().pin_memory(), u_v.cpu().pin_memory(), u_len.cpu().pin_memory()
    h_th = u_th.cpu().pin_memory()
    h_Y = u_Y.cpu().pin_memory()
    srcs = (h_lane, h_p, h_v, h_len, h_th, h_Y)
    bufs = [tuple(torch.empty_like(t) for t in (u_lane, u_p, u_v, u_len, u_th, u_Y)) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    out_th = torch.empty(s_th.shape).pin_memory()
    out_hist = torch.empty(hist.shape, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_lane, h_p, h_v, h_len, h_th, h_Y))
    d2h = out_th.numel() * 4 + out_hist.numel() * 8
    lib.idm_set_profiling(h, 0)
    barrier()
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    copy_stream.wait_event(e2)  # no copy starts before the timed region

    def issue_copy(i):
        b = i % 2
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(free[b])  # the step two back is done with buffer b
            for dst, src in zip(bufs[b], srcs):
                dst.copy_(src, non_blocking=True)
            ready[b].record(copy_stream)

    issue_copy(0)
    for i in range(e2e_steps):
        b = i % 2
        if i + 1 < e2e_steps:
            issue_copy(i + 1)
        stream.wait_event(ready[b])
        step(*bufs[b])
        free[b].record(stream)
        out_th.copy_(s_th, non_blocking=True)
        out_hist.copy_(hist, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e2.elapsed_time(e3))
    del h_Y, bufs
    return ms, h2d, d2h


# Algorithmic FLOPs of one training sample of the initializer (forward,
# input-gradient of layers 2-4, weight gradients; the 5-wide output layer
# counted at its real width).
MLP_FWD_FLOP = 2 * (80 * 256 + 256 * 256 + 256 * 256 + 256 * 5)
MLP_TRAIN_FLOP = 2 * MLP_FWD_FLOP + 2 * (256 * 5 + 2 * 256 * 256)


def time_to_fit(a, dev):
    """Initializer experiment: train the network on simulated noisy 20-step
    prefixes, then fit a 200K-vehicle scene (2,000 lanes x 100, 100 steps,
    every step observed, noise 0.5 m) from the learned and from the plain
    initial guess with the same Adam schedule; report iterations and wall
    time until the fitted trajectory is within --rmse-target (RMSE against
    the noise-free truth) and the network's training throughput."""
    import torch
    from paper_2412_16750_gb300 import api, synth, tune
    cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20241216 + 3)
    out = {}

    # ---- training set ------------------------------------------------------
    tr = synth.config3_train(n_lanes=a.init_train_lanes)
    Ntr = int(tr["lane_off"][-1])
    scene = api.Scene.from_lane_off(cu(tr["lane_off"], torch.int32), cu(tr["length"]), 100)
    th = cu(tr["theta_true"])
    p0, v0 = cu(tr["p_init"]), cu(tr["v_init"])
    del tr
    P = api.simulate(th, p0, v0, scene, 20, DT)
    Y = P[1:]
    Y.add_(0.5 * torch.randn(Y.shape, device=dev, generator=gen))
    perm = torch.randperm(Ntr, device=dev, generator=gen).to(torch.int32)
    X, lab = api.mlp_features(scene, p0, v0, 20, DT, Y, 1, perm=perm, theta=th)
    del P, Y, perm, th, p0, v0, scene
    torch.cuda.empty_cache()
    net = api.Mlp(max_batch=a.mlp_batch, weights=synth.mlp_init(0))
    n_steps = a.mlp_epochs * (Ntr // a.mlp_batch)
    net.train(X, lab, a.mlp_batch, 20, 2e-3, 2e-3)          # warm-up (modules, caches)
    net.set_weights(synth.mlp_init(0))
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    hist = net.train(X, lab, a.mlp_batch, n_steps, 2e-3, 2e-4)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    rc, bits = net.status()
    if rc != 0:
        raise RuntimeError("initializer status %d bits %d" % (rc, bits))
    samples = n_steps * a.mlp_batch
    label_mean = lab.double().mean(0).cpu().numpy()
    label_var = float(lab.double().var(0).mean().item())     # MSE of the best input-free guess
    del X, lab
    torch.cuda.empty_cache()
    out["mlp"] = {"train_samples": Ntr, "epochs": a.mlp_epochs, "batch": a.mlp_batch, "steps": n_steps,
                  "train_s": train_ms / 1e3, "samples_per_s": samples / (train_ms / 1e3),
                  "tflops": MLP_TRAIN_FLOP * samples / (train_ms / 1e3) / 1e12,
                  "flop_per_sample": MLP_TRAIN_FLOP,
                  "loss_first": float(hist[:10].mean().item()), "loss_last": float(hist[-10:].mean().item()),
                  "label_variance": label_var}

    # ---- fit scene ---------------------------------------------------------------
    fs = synth.config3_fit()
    N, K = int(fs["lane_off"][-1]), fs["K"]
    scene = api.Scene.from_lane_off(cu(fs["lane_off"], torch.int32), cu(fs["length"]), 100)
    th_true = cu(fs["theta_true"])
    p0, v0 = cu(fs["p_init"]), cu(fs["v_init"])
    P = api.simulate(th_true, p0, v0, scene, K, DT)
    clean = P[1:].contiguous()
    Y = (clean + 0.5 * torch.randn(clean.shape, device=dev, generator=gen)).contiguous()
    plain = cu(synth.plain_init(N))
    ctx = api.Context()
    th_buf = torch.empty_like(plain)
    # kernel shape for this problem size (autotuner, cached per GPU), timed on
    # a short fit: the shape also decides the fit's form and tape depth
    sig = tune.signature(100, N, K, 1, kind="fit-20")
    scratch = plain.clone()
    shape, shape_src, _ = tune.tuned(ctx, lambda c: api.fit(scratch, p0, v0, scene, K, DT, Y, 1, 20, ctx=c), 100,
                                     sig, repeats=3)

    def timed(fn):
        e0, e1 = ev(), ev()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    # per-iteration time of the fit (graph captured by the first call)
    for _ in range(2):
        th_buf.copy_(plain)
        _, fit_ms = timed(lambda: api.fit(th_buf, p0, v0, scene, K, DT, Y, 1, a.fit_iters, ctx=ctx))
    ms_iter = fit_ms / a.fit_iters
    fit_form = ctx.last_fit_form()

    def first_below(ev_hist):
        rmse = np.sqrt(ev_hist.cpu().numpy() / N)
        hit = np.nonzero(rmse <= a.rmse_target)[0]
        return (int(hit[0]) if hit.size else None), rmse

    th_buf.copy_(plain)
    _, ev_plain = api.fit(th_buf, p0, v0, scene, K, DT, Y, 1, a.fit_iters, ctx=ctx, eval_targets=clean)
    it_plain, rmse_plain = first_below(ev_plain)
    # learned initial guess: features of the first 20 observations + inference
    for _ in range(2):
        th_buf.copy_(plain)
        _, init_ms = timed(lambda: net.predict_params(
            api.mlp_features(scene, p0, v0, K, DT, Y, 1), th_buf))
    # label MSE of the learned guess on this (held-out) scene, in the
    # network's normalized units, beside that of the training-label mean
    lo_t = torch.tensor(synth.BOX_LO, device=dev, dtype=torch.float64)[:, None]
    hi_t = torch.tensor(synth.BOX_HI, device=dev, dtype=torch.float64)[:, None]
    _, lab_fit = api.mlp_features(scene, p0, v0, K, DT, Y, 1, theta=th_true)
    lab_fit = lab_fit.double().t()
    pred_norm = (th_buf[:5].double() - lo_t) / (hi_t - lo_t)
    label_mse = {"network": float(((pred_norm - lab_fit) ** 2).mean().item()),
                 "training_mean": float(((torch.as_tensor(label_mean, device=dev)[:, None] - lab_fit) ** 2)
                                        .mean().item())}
    del lab_fit, pred_norm
    _, ev_learned = api.fit(th_buf, p0, v0, scene, K, DT, Y, 1, a.fit_iters, ctx=ctx, eval_targets=clean)
    it_learned, rmse_learned = first_below(ev_learned)
    ctx.set_event_counting(True)
    ctx.event_counts()
    api.simulate(th_buf, p0, v0, scene, K, DT, ctx=ctx)
    events_learned = ctx.event_counts()
    ctx.set_event_counting(False)
    # ablation: every vehicle starts at the mean of the training labels (what
    # the network could know without looking at the trajectories)
    lo, hi = np.array(synth.BOX_LO), np.array(synth.BOX_HI)
    mean_th = synth.plain_init(N)
    mean_th[:5] = (lo + (hi - lo) * label_mean)[:, None]
    th_buf.copy_(cu(mean_th))
    _, ev_mean = api.fit(th_buf, p0, v0, scene, K, DT, Y, 1, a.fit_iters, ctx=ctx, eval_targets=clean)
    it_mean, rmse_mean = first_below(ev_mean)
    wall = lambda it, extra: (extra + it * ms_iter) / 1e3 if it is not None else None
    out["fit"] = {"workload": "2000 lanes x 100 vehicles (200K), 100 steps, every step observed, noise 0.5 m; "
                              "Adam %d iterations, lr 0.1 -> 0.01" % a.fit_iters,
                  "rmse_target_m": a.rmse_target, "ms_per_iteration": ms_iter, "fit_form": fit_form,
                  "shape": {"vpt": shape[0], "warps_per_segment": shape[1], "ckpt_interval": shape[2],
                            "warps_per_block": shape[3], "source": shape_src},
                  "plain": {"iterations": it_plain, "seconds": wall(it_plain, 0.0),
                            "rmse_m_at": {str(i): float(rmse_plain[i]) for i in (0, 10, 50, 100, a.fit_iters - 1)
                                          if i < a.fit_iters}},
                  "learned": {"iterations": it_learned, "seconds": wall(it_learned, init_ms),
                              "init_ms": init_ms, "label_mse_held_out": label_mse,
                              "rmse_m_at": {str(i): float(rmse_learned[i])
                                            for i in (0, 10, 50, 100, a.fit_iters - 1) if i < a.fit_iters}},
                  "events_learned_fit": events_learned,
                  "training_mean_ablation": {"iterations": it_mean, "seconds": wall(it_mean, 0.0),
                                             "rmse_m_at": {str(i): float(rmse_mean[i])
                                                           for i in (0, 10, 50, 100, a.fit_iters - 1)
                                                           if i < a.fit_iters}}}
    ctx.close()
    return out, net


def long_horizon(a, dev, net):
    """2M vehicles, 3,000 steps: fit (v0, T, s0, a_max, b) on noisy
    observations of steps 1..2,000 from the learned initial guess with
    --long-iters Adam iterations (checkpoints every 45 steps, about
    sqrt(2000)), then simulate all 3,000 steps with the fitted parameters
    and score steps 2,001..3,000 against the truth; sampled lanes are
    re-simulated by the FP64 oracle with the same fitted parameters."""
    import torch
    import oracle
    from paper_2412_16750_gb300 import api, synth
    cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device=dev)
    stream = torch.cuda.current_stream(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20241216 + 4)
    K_fit, K_all, C = 2000, 3000, 45
    sc = synth.make_scene([100] * a.long_lanes, synth.rng_for(4))
    N = int(sc["lane_off"][-1])
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    scene = api.Scene.from_lane_off(cu(sc["lane_off"], torch.int32), cu(sc["length"]), 100)
    p0, v0 = cu(sc["p_init"]), cu(sc["v_init"])
    ctx = api.Context(ckpt_interval=C)
    truth = api.simulate(cu(sc["theta_true"]), p0, v0, scene, K_all, DT, ctx=ctx)
    Y = (truth[1:K_fit + 1] + 0.5 * torch.randn((K_fit, N), device=dev, generator=gen)).contiguous()
    th = cu(synth.plain_init(N))
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    net.predict_params(api.mlp_features(scene, p0, v0, K_fit, DT, Y, 1), th)
    e[1].record(stream)
    hist = api.fit(th, p0, v0, scene, K_fit, DT, Y, 1, a.long_iters, ctx=ctx)
    e[2].record(stream)
    pred = api.simulate(th, p0, v0, scene, K_all, DT, ctx=ctx)
    e[3].record(stream)
    torch.cuda.synchronize()
    rc, flags = ctx.status()
    if rc != 0:
        raise RuntimeError("long-horizon status %d flags %d" % (rc, flags))
    peak = torch.cuda.max_memory_allocated(dev)
    ws = lib_workspace(ctx, scene, K_fit)
    ctx.set_event_counting(True)
    ctx.event_counts()
    api.simulate(th, p0, v0, scene, K_all, DT, ctx=ctx)
    events = ctx.event_counts()
    ctx.set_event_counting(False)
    err = (pred[K_fit + 1:] - truth[K_fit + 1:]).double()
    rmse_pred = float(torch.sqrt((err * err).mean()).item())
    err_fit = (pred[1:K_fit + 1] - truth[1:K_fit + 1]).double()
    rmse_fit = float(torch.sqrt((err_fit * err_fit).mean()).item())
    # FP64 oracle on sampled lanes with the GPU's fitted parameters
    lanes = np.linspace(0, a.long_lanes - 1, 8).astype(int)
    th_h = th.double().cpu().numpy()
    pred_h = None
    worst = 0.0
    for l in lanes:
        i0, i1 = int(sc["lane_off"][l]), int(sc["lane_off"][l + 1])
        lo = np.array([0, i1 - i0], dtype=np.int32)
        P, _ = oracle.forward(lo, sc["length"][i0:i1], th_h[:, i0:i1], sc["p_init"][i0:i1], sc["v_init"][i0:i1],
                              K_all, DT, A_MIN)
        pred_h = pred[:, i0:i1].double().cpu().numpy()
        worst = max(worst, float(np.max(np.abs(pred_h - P))))
    out = {"workload": "%d lanes x 100 vehicles (%.1fM), fit steps 1-%d (noise 0.5 m), predict steps %d-%d; "
                       "learned initial guess + %d Adam iterations, checkpoints every %d steps"
                       % (a.long_lanes, N / 1e6, K_fit, K_fit + 1, K_all, a.long_iters, C),
           "init_ms": e[0].elapsed_time(e[1]), "fit_s": e[1].elapsed_time(e[2]) / 1e3,
           "predict_ms": e[2].elapsed_time(e[3]),
           "fit_vehicle_steps_per_s": a.long_iters * N * K_fit / (e[1].elapsed_time(e[2]) * 1e-3),
           "rmse_fit_window_m": rmse_fit, "rmse_prediction_m": rmse_pred,
           "rmse_vs_noisy_targets_m": {"before_first_update": math.sqrt(float(hist[0].item()) / N),
                                       "before_last_update": math.sqrt(float(hist[-1].item()) / N)},
           "oracle_check": {"lanes": len(lanes), "max_abs_diff_m": worst, "steps": K_all},
           "events_fitted": events,
           "peak_hbm_gb": {"torch_allocated": peak / 1e9, "library_workspace": ws / 1e9}}
    ctx.close()
    return out


def lib_workspace(ctx, scene, K):
    from paper_2412_16750_gb300 import lib
    return lib.idm_workspace_bytes(ctx.handle, scene.c(), lib.make_sim(K, DT, A_MIN))


def batched(a, dev):
    """Batched uneven scenarios: 4,096 scenarios (lanes U[1,64], vehicles per
    lane U[2,200], horizons U[50,500], observed every 10th step) fitted
    together, one forward and one adjoint launch per Adam iteration, the whole
    fit one CUDA graph; kernel shape chosen by the autotuner (cached)."""
    import torch
    from paper_2412_16750_gb300 import api, synth, tune
    cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device=dev)
    stream = torch.cuda.current_stream(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20241216 + 2)
    sc = synth.config2(a.batch_scen)
    N = int(sc["lane_off"][-1])
    b = api.Batch(sc["scen_lane_off"], sc["K"], sc["dt"], sc["obs_stride"], sc["lane_off"], sc["length"], A_MIN)
    th_true = cu(sc["theta_true"])
    p0, v0 = cu(sc["p_init"]), cu(sc["v_init"])
    ctx = api.Context()
    # clean observed targets of every scenario (rows j*10 of its trajectory block)
    traj = api.batch_forward(th_true, p0, v0, b, ctx=ctx)
    nv = np.diff(b.veh_off)
    clean = torch.empty(int(b.tgt_off[-1]), device=dev)
    for q in range(b.n_scen):
        K, st, n = int(b.K[q]), int(b.obs_stride[q]), int(nv[q])
        blk = traj[b.traj_off[q]:b.traj_off[q + 1]].view(K + 1, n)
        clean[b.tgt_off[q]:b.tgt_off[q + 1]].view(-1, n).copy_(blk[st::st][:K // st])
    del traj
    torch.cuda.empty_cache()
    Y = clean + 0.5 * torch.randn(clean.shape, device=dev, generator=gen)
    plain = cu(synth.plain_init(N))
    max_lane = int(np.diff(sc["lane_off"]).max())
    sig = tune.signature(max_lane, N, float(np.mean(sc["K"])), 10, kind="batch")
    run = lambda c: api.batch_loss_grad(plain, p0, v0, b, Y, ctx=c)
    shape, how, timings = tune.tuned(ctx, run, max_lane, sig, repeats=2)
    units = int(np.sum(nv.astype(np.int64) * b.K.astype(np.int64)))    # vehicle-steps per forward
    th = torch.empty_like(plain)
    for _ in range(2):                                                  # first call captures the graph
        th.copy_(plain)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hist, _ = api.batch_fit(th, p0, v0, b, Y, a.batch_iters, ctx=ctx)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_iter = e0.elapsed_time(e1) / a.batch_iters
    fit_form = ctx.last_fit_form()
    rc, flags = ctx.status()
    if rc != 0:
        raise RuntimeError("batched status %d flags %d" % (rc, flags))
    ctx.set_event_counting(True)
    ctx.event_counts()
    api.batch_forward(th, p0, v0, b, ctx=ctx)
    events = ctx.event_counts()
    ctx.set_event_counting(False)
    _, tot_clean, _, _, _ = api.batch_loss_grad(th, p0, v0, b, clean, ctx=ctx)
    _, tot0, _, _, _ = api.batch_loss_grad(plain, p0, v0, b, clean, ctx=ctx)
    out = {"workload": sc["name"], "vehicles": N, "lanes": int(sc["scen_lane_off"][-1]),
           "vehicle_steps_per_iteration": units, "iterations": a.batch_iters, "ms_per_iteration": ms_iter,
           "vehicle_steps_per_s": units / (ms_iter * 1e-3), "fit_form": fit_form,
           "launches_per_iteration": 3 if fit_form == "graph" else None,
           "shape": {"vpt": shape[0], "warps_per_segment": shape[1], "ckpt_interval": shape[2],
                     "warps_per_block": shape[3], "source": how, "candidates_timed": len(timings)},
           "events_fitted": events,
           "rmse_vs_clean_m": {"initial": math.sqrt(float(tot0.item()) / N),
                               "after_%d_iterations" % a.batch_iters: math.sqrt(float(tot_clean.item()) / N)}}
    ctx.close()
    return out


# Algorithmic bytes per trajectory-step of one fit iteration of the
# reconstruction mode: forward reads dp, dv and the observation row (16 B)
# and writes the tape (32 B); the adjoint reads the tape, dp, dv and four Adam
# moments (56 B) and writes dp, dv and the moments (24 B).
RECON_BYTES_PER_STEP = 16 + 32 + 56 + 24


def reconstruction(a, dev):
    """Single-trajectory filtering and reconstruction (Sec. IV-A; settings
    and metrics of Sec. V-B) on the synthetic stand-ins of the paper's two
    data sets: every trajectory fitted with 500 Adam iterations (lr 0.1 ->
    0.01) from the paper's starting point, all trajectories in one launch."""
    import torch
    from oracle import recon as R
    from paper_2412_16750_gb300 import api, synth
    cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device=dev)
    stream = torch.cuda.current_stream(dev)
    peaks, _ = measured_peaks()
    out = {}
    for k, (name, spec, paper_s) in enumerate((("filtering", synth.FILTER_SPEC, 0.308),
                                               ("reconstruction", synth.RECON_SPEC, 0.164))):
        rng = np.random.default_rng(synth.SEED_BASE + 50 + k)
        off, t, p = synth.recon_observations(spec["n"], spec["dur"], rng, dense=spec.get("dense"),
                                             gap_min=spec.get("gap_min", 1.0),
                                             gap_mean_extra=spec.get("gap_mean_extra", 1.0), noise=spec["noise"])
        ctx = api.Context()
        r = api.Recon(cu(off, torch.int32), cu(t), cu(p), spec["dt"], A_MIN, ctx=ctx)
        th0, dp0, dv0 = r.init_vars()
        m0 = r.metrics(th0, dp0, dv0).cpu().numpy()
        th, dp, dv = th0.clone(), dp0.clone(), dv0.clone()
        r.fit(th, dp, dv, 3)                                   # warm-up
        th.copy_(th0), dp.copy_(dp0), dv.copy_(dv0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hist = r.fit(th, dp, dv, a.recon_iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rc, flags = ctx.status()
        if rc != 0:
            raise RuntimeError("reconstruction status %d flags %d" % (rc, flags))
        m1 = r.metrics(th, dp, dv).cpu().numpy()
        K = r.K.cpu().numpy()[:r.N].astype(np.int64)
        steps = int(K.sum())
        h = hist.cpu().numpy()
        gbs = RECON_BYTES_PER_STEP * steps * a.recon_iters / (ms * 1e-3) / 1e9
        # the oracle's fit of a bounded sample of the same trajectories
        n_cpu = 8 if name == "reconstruction" else 16
        sel = np.linspace(0, spec["n"] - 1, n_cpu).astype(int)
        offs = np.concatenate([[0], np.cumsum(np.diff(off)[sel])]).astype(np.int32)
        idx = np.concatenate([np.arange(off[i], off[i + 1]) for i in sel])
        ok = R.nearest_steps(t[idx], spec["dt"])
        Ks = R.horizons(offs, ok)
        p0s, v0s = R.init_state(offs, t[idx], p[idx])
        ths = np.array(api.RECON_INIT)[:, None].repeat(n_cpu, 1)
        km = int(Ks.max())
        tc = time.perf_counter()
        R.fit(Ks, np.full((km, n_cpu), 10.0), np.zeros((km, n_cpu)), ths, p0s, v0s, spec["dt"], offs, ok, p[idx],
              a.recon_iters, 0.1, 0.01, api.RECON_BOX_LO, api.RECON_BOX_HI, A_MIN)
        cpu_s = (time.perf_counter() - tc) / n_cpu
        out[name] = {
            "workload": "%d trajectories, %s, durations U[%g, %g] s, noise %g m, dt %g s" % (
                spec["n"], ("every %g s" % spec["dense"]) if spec.get("dense") else
                ("intervals %g s + Exp(mean %g s)" % (spec["gap_min"], spec["gap_mean_extra"])),
                spec["dur"][0], spec["dur"][1], spec["noise"], spec["dt"]),
            "observations": int(off[-1]), "k_max": r.k_max, "trajectory_steps": steps,
            "iterations": a.recon_iters, "fit_ms": ms, "s_per_trajectory": ms * 1e-3 / spec["n"],
            "paper_s_per_trajectory": paper_s,
            "trajectory_steps_per_s": steps * a.recon_iters / (ms * 1e-3),
            "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
            "roofline": {"kernel": "recon_fit_kernel (all iterations in one launch)", "bound": "hbm",
                         "achieved": gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                         "bytes_per_trajectory_step": RECON_BYTES_PER_STEP,
                         "note": "one serial chain per trajectory: with few trajectories (filtering) the kernel is "
                                 "latency-bound below this roof"},
            "us_per_step_of_longest": ms * 1e3 / (a.recon_iters * r.k_max),
            "gpu_launches": 1,
            "loss": {"initial": float(h[0]), "final": float(h[-1])},
            "metrics_initial": {"pos": float(m0[0]), "acc_mean": float(m0[1]), "acc_std": float(m0[2]),
                                "imp": float(m0[3])},
            "metrics_fitted": {"pos": float(m1[0]), "acc_mean": float(m1[1]), "acc_std": float(m1[2]),
                               "imp": float(m1[3])},
            "paper_metrics": {"filtering": "Pos 0.08%, Acc 0.5/0.5, Imp 0% (NGSIM)",
                              "reconstruction": "Pos 0.13%, Acc 0.3/1.1, Imp 0% (Singapore)"}[name],
            "cpu_oracle_s_per_trajectory": cpu_s, "cpu_oracle_sample": "%d trajectories, 1 core" % n_cpu,
        }
        ctx.close()
        del r, th0, dp0, dv0, th, dp, dv
        torch.cuda.empty_cache()
    return out


def cpu_gpu_crossover(a, dev):
    """Time of one loss + gradient (forward and adjoint over K = 100 steps)
    per vehicle count on the multi-threaded CPU backend (every host core)
    and on the GPU, lanes of 100 vehicles: the comparison of the paper's
    Fig. 1 (CPU faster for small counts, GPU beyond about 20K vehicles)."""
    import torch
    from paper_2412_16750_gb300 import api, build, cpu, synth
    build.build_cpu()
    K, s = 100, 1
    stream = torch.cuda.current_stream(dev)
    rows = []
    for N in (100, 300, 1000, 4000, 16000, 64000, 256000, 1000000, 2000000):
        sc = synth.make_scene([min(100, N)] * max(1, N // 100), np.random.default_rng(synth.SEED_BASE + 60))
        n = len(sc["length"])
        th = synth.plain_init(n)
        Y = synth.f32(np.random.default_rng(1).normal(0.0, 1.0, size=(K, n)) + sc["p_init"][None, :] +
                      np.arange(1, K + 1)[:, None] * 1.5)
        cs = cpu.Scene(sc["lane_off"], sc["length"])
        cpu.idm_cpu_loss_grad(th, sc["p_init"], sc["v_init"], cs, K, DT, Y, s, A_MIN)
        reps = max(1, min(20, int(2e6 // n)))
        t0 = time.perf_counter()
        for _ in range(reps):
            cpu.idm_cpu_loss_grad(th, sc["p_init"], sc["v_init"], cs, K, DT, Y, s, A_MIN)
        cpu_ms = (time.perf_counter() - t0) * 1e3 / reps
        cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device=dev)
        ctx = api.Context()
        scene = api.Scene.from_lane_off(cu(sc["lane_off"], torch.int32), cu(sc["length"]))
        tg, pg, vg, Yg = cu(th), cu(sc["p_init"]), cu(sc["v_init"]), cu(Y)
        for _ in range(3):
            api.loss_grad(tg, pg, vg, scene, K, DT, Yg, s, A_MIN, ctx=ctx)
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            api.loss_grad(tg, pg, vg, scene, K, DT, Yg, s, A_MIN, ctx=ctx)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        gpu_ms = sorted(ts)[len(ts) // 2]
        ctx.close()
        rows.append({"vehicles": n, "cpu_ms": cpu_ms, "gpu_ms": gpu_ms,
                     "cpu_ms_per_timestep": cpu_ms / K, "gpu_ms_per_timestep": gpu_ms / K})
    cross = next((r["vehicles"] for r in rows if r["gpu_ms"] < r["cpu_ms"]), None)
    return {"workload": "loss + gradient, K = 100 steps, lanes of 100 vehicles, every step observed",
            "cpu_threads": cpu.max_threads(), "rows": rows, "gpu_faster_from_vehicles": cross,
            "paper": "Fig. 1: CPU (16 threads) faster below ~20K vehicles, GPU beyond"}


def prediction(a, dev):
    """Training-free prediction with lane geometry (Sec. IV-B, V-C) on a
    synthetic stand-in for the Waymo Open Motion validation set: assign and
    project 1 s of history (11 frames at 10 Hz) onto lane centre lines, fit
    the IDM parameters on the 10 history steps (500 Adam iterations), roll out
    80 steps (8 s), project back and score against the true future."""
    import torch
    from paper_2412_16750_gb300 import api, synth
    cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device=dev)
    stream = torch.cuda.current_stream(dev)
    sc = synth.prediction_scenes(a.pred_scen, np.random.default_rng(synth.SEED_BASE + 70))
    peaks, _ = measured_peaks()
    H, Fn = sc["n_hist"], sc["n_fut"]
    N = sc["x"].shape[1]
    ctx = api.Context()
    L = api.Lanes(cu(sc["pt_off"], torch.int32), cu(sc["px"]), cu(sc["py"]), ctx=ctx)
    xh, yh = cu(sc["x"][:H]), cu(sc["y"][:H])
    lo, hi = cu(sc["lane_lo"], torch.int32), cu(sc["lane_hi"], torch.int32)
    xt, yt = cu(sc["x"][H:]), cu(sc["y"][H:])
    api.predict_rollout(L, xh, yh, lo, hi, sc["dt"], Fn, 3, ctx=ctx, tune=True)   # warm-up; tunes the fit's shape
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    lane, _, _ = L.project(xh[H - 1], yh[H - 1], lo, hi, want=("lane",))
    _, s_hist, _ = L.project(xh, yh, lane.view(N), None, want=("s",))
    ev[1].record(stream)
    out = api.predict_rollout(L, xh, yh, lo, hi, sc["dt"], Fn, a.pred_iters, ctx=ctx)
    perm = out["perm"]
    tx, ty = torch.empty_like(xt), torch.empty_like(yt)
    from paper_2412_16750_gb300 import lib
    lib.idm_gather_rows(ctx.handle, N, Fn, perm, xt, tx, stream)
    lib.idm_gather_rows(ctx.handle, N, Fn, perm, yt, ty, stream)
    ade, fde, sums = api.displacement(out["x"], out["y"], tx, ty, 2.0, ctx=ctx)
    ev[2].record(stream)
    torch.cuda.synchronize()
    rc, flags = ctx.status()
    if rc != 0:
        raise RuntimeError("prediction status %d flags %d" % (rc, flags))
    sums = sums.cpu().numpy()
    seg_assign = int(np.sum((sc["pt_off"][sc["lane_hi"]] - sc["pt_off"][sc["lane_lo"]]) - (sc["lane_hi"] - sc["lane_lo"])))
    seg_proj = int(H * np.sum(sc["pt_off"][out["lane"].cpu().numpy() + 1] - sc["pt_off"][out["lane"].cpu().numpy()] - 1))
    proj_ms = ev[0].elapsed_time(ev[1])
    total_ms = ev[1].elapsed_time(ev[2])
    res = {"workload": "%d scenarios, lanes U[2, 8] per scenario (300 m arcs sampled every 2 m), agents U[1, 6] per "
                       "lane, 1 s history at 10 Hz, 8 s future" % a.pred_scen,
           "agents": N, "lanes": sc["n_lanes"], "fit_iterations": a.pred_iters,
           "pipeline_ms": total_ms, "ms_per_scenario": total_ms / a.pred_scen,
           "projection_ms": proj_ms, "projection_segments": seg_assign + seg_proj,
           "projection_segments_per_s": (seg_assign + seg_proj) / (proj_ms * 1e-3),
           "projection_roofline": {"kernel": "project_kernel", "bound": "alu",
                                   "achieved": 15.0 * (seg_assign + seg_proj) / (proj_ms * 1e-3) / 1e9,
                                   "peak": alu_peak_ginst(peaks.get("sm_max_mhz", 2070.0),
                                                          torch.cuda.get_device_properties(dev).multi_processor_count),
                                   "unit": "Ginstr/s (FP32 pipe)",
                                   "ops_per_segment": 15,
                                   "note": "FP32 operations of one segment distance (direction, clamped parameter, "
                                           "foot point, squared distance, compare); two projection launches"},
           "ade_m": float(sums[0] / N), "fde_m": float(sums[1] / N), "miss_rate_2m": float(sums[2] / N),
           "final_loss": float(out["loss"][-1].item()), "fit_shape": list(ctx.tuning),
           "fit_form": ctx.last_fit_form(),
           "paper": "WOMD validation: minADE 7.862 m, minFDE 15.668 m, miss rate 0.586 (Table II)"}
    ctx.close()
    return res


def run_gpu(a, rank, world, local_rank):
    import torch
    from paper_2412_16750_gb300 import api, lib, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    if a.pred_only:
        if rank == 0:
            print(json.dumps({"prediction": prediction(a, dev)}), flush=True)
        return 0
    if a.crossover_only:
        if rank == 0:
            print(json.dumps({"cpu_gpu_crossover": cpu_gpu_crossover(a, dev)}), flush=True)
        return 0
    if a.recon_only:
        if rank == 0:
            print(json.dumps({"reconstruction": reconstruction(a, dev)}), flush=True)
        return 0
    if a.batched_only:
        if rank == 0:
            print(json.dumps({"batched": batched(a, dev)}), flush=True)
        return 0
    if a.init_only:
        if rank == 0:
            ttf, net = time_to_fit(a, dev)
            print(json.dumps({"time_to_fit": ttf}), flush=True)
        return 0
    if a.long_only:
        if rank == 0:
            ttf, net = time_to_fit(a, dev)
            print(json.dumps({"time_to_fit": ttf, "long_horizon": long_horizon(a, dev, net)}), flush=True)
        return 0

    # ---- this rank's share of the job's scene, unsorted arrival order -----
    # The job's scene has world x --lanes lanes of --per-lane vehicles; lanes
    # are independent, so each rank takes a contiguous lane range balanced by
    # vehicles x steps (dist.lane_shards) and the ranks exchange only the FP64
    # loss history of each step's fit (one all-reduce).
    from paper_2412_16750_gb300 import dist as idm_dist
    L_job = a.lanes * world
    l0, l1 = idm_dist.lane_shards(synth.lane_offsets([a.per_lane] * L_job), world)[rank]
    rng = synth.rng_for(1, l0)                  # seeded by the shard's first lane
    counts = [a.per_lane] * (l1 - l0)
    sc = synth.make_scene(counts, rng)
    N = int(sc["lane_off"][-1])
    L = l1 - l0
    K = a.K
    ctx = api.Context(vpt=a.vpt, warps_per_segment=a.G, ckpt_interval=a.ckpt, warps_per_block=a.wpb)
    cu = lambda x, d=torch.float32: torch.as_tensor(np.ascontiguousarray(x), dtype=d, device=dev)
    scene_sorted = api.Scene.from_lane_off(cu(sc["lane_off"], torch.int32), cu(sc["length"]), a.per_lane)
    th_true = cu(sc["theta_true"])
    p_sorted, v_sorted = cu(sc["p_init"]), cu(sc["v_init"])
    gen = torch.Generator(device=dev)
    gen.manual_seed(20241216 + 1000 * l0)
    traj = api.simulate(th_true, p_sorted, v_sorted, scene_sorted, K, DT, A_MIN, ctx=ctx)
    Y_sorted = traj[1:]
    Y_sorted.add_(0.5 * torch.randn(Y_sorted.shape, device=dev, generator=gen))
    order = torch.as_tensor(rng.permutation(N), device=dev)
    lane_id = torch.repeat_interleave(torch.arange(L, device=dev, dtype=torch.int32),
                                      torch.as_tensor(np.diff(sc["lane_off"]), device=dev))
    # arrival-order inputs (device resident)
    u_lane = lane_id[order].contiguous()
    u_p = p_sorted[order].contiguous()
    u_v = v_sorted[order].contiguous()
    u_len = scene_sorted.length[order].contiguous()
    u_th = cu(synth.plain_init(N))[:, order].contiguous()
    u_Y = Y_sorted[:, order].contiguous()
    del traj, Y_sorted
    torch.cuda.empty_cache()

    # ---- preallocated step buffers ---------------------------------------
    perm = torch.empty(N, dtype=torch.int32, device=dev)
    lane_off = torch.empty(L + 1, dtype=torch.int32, device=dev)
    mx = torch.zeros(1, dtype=torch.int32, device=dev)
    s_p = torch.empty(N, device=dev)
    s_v = torch.empty(N, device=dev)
    s_len = torch.empty(N, device=dev)
    s_th = torch.empty((6, N), device=dev)
    s_Y = torch.empty((K, N), device=dev)
    hist = torch.zeros(a.iters, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = ctx.handle
    lib.idm_set_profiling(h, 1)
    scene_c = lib.idm_scene_t(L, N, a.per_lane, lane_off.data_ptr(), s_len.data_ptr())
    params_c = lib.make_params(s_th)
    sim_c = lib.make_sim(K, DT, A_MIN)

    def reduce_hist():
        # the job's loss history: the shards' FP64 histories summed (the one
        # data-path collective; lanes never interact)
        if dist is not None:
            dist.all_reduce(hist, op=dist.ReduceOp.SUM)

    def step(in_lane, in_p, in_v, in_len, in_th, in_Y):
        lib.idm_layout(h, N, L, in_lane, in_p, perm, lane_off, mx, stream)
        lib.idm_gather(h, N, perm, [in_p, in_v, in_len] + [in_th[q] for q in range(6)],
                       [s_p, s_v, s_len] + [s_th[q] for q in range(6)], stream)
        lib.idm_gather_rows(h, N, K, perm, in_Y, s_Y, stream)
        lib.idm_fit(h, scene_c, params_c, s_p, s_v, sim_c, s_Y, 1, a.iters, 0.1, 0.01, synth.BOX_LO, synth.BOX_HI,
                    hist, stream)
        reduce_hist()

    launches_per_step = 4 + 1 + 1 + 3 + 3 * a.iters  # layout 4, gather 1, rows 1, prep 3, 3 per iteration

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def measure(steps, warmup, sample_clocks):
        """warmup untimed steps, then `steps` timed ones (device-resident
        inputs); adjoint and forward launch times from the fit graph's events."""
        for _ in range(warmup):
            step(u_lane, u_p, u_v, u_len, u_th, u_Y)
        torch.cuda.synchronize()
        rc, flags = ctx.status()
        if rc != 0:
            raise RuntimeError("device status %d flags %d: %s" % (rc, flags, lib.idm_last_error(h)))
        clocks = ClockSampler(local_rank) if sample_clocks else None
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        fwd_ms = bwd_ms = 0.0
        n_fit_iters = 0
        e0.record(stream)
        for _ in range(steps):
            step(u_lane, u_p, u_v, u_len, u_th, u_Y)
            f, b, n = lib.idm_phase_times(h, stream)  # syncs the stream: per-launch event times of this step
            fwd_ms += f
            bwd_ms += b
            n_fit_iters += n
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1))
        return {"ms": ms, "fwd_avg_ms": fwd_ms / max(n_fit_iters, 1), "bwd_avg_ms": bwd_ms / max(n_fit_iters, 1),
                "clocks": clk}

    peaks, peak_kind = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    units_per_step = a.iters * N * K

    # ---- timed: device-resident inputs, the stated checkpoint interval ------
    m = measure(a.steps, a.warmup, True)
    ms = m["ms"]
    final_loss = float(hist[-1].item()) / (N * world)

    # ---- timed: end to end from pinned host memory --------------------------
    e2e_steps = a.e2e_steps if a.e2e_steps is not None else a.steps
    ms_e2e, h2d, d2h = None, 0, 0
    if e2e_steps > 0:
        ms_e2e, h2d, d2h = run_e2e(a, e2e_steps, step, barrier, max_over_ranks, stream, dev, u_lane, u_p, u_v, u_len,
                                   u_th, u_Y, s_th, hist, h, lib)
        rc, flags = ctx.status()
        if rc != 0:
            raise RuntimeError("device status %d flags %d after e2e" % (rc, flags))

    value = world * units_per_step * a.steps / (ms * 1e-3)
    e2e_value = world * units_per_step * e2e_steps / (ms_e2e * 1e-3) if ms_e2e else None
    roofline = adjoint_roofline(N, K, a.ckpt, m["bwd_avg_ms"], n_sm, peaks, peak_kind)

    # ---- the same step at the tuned checkpoint interval (labelled variant) ----
    tuned = None
    if a.tuned_ckpt and a.tuned_ckpt != a.ckpt and a.tuned_steps > 0:
        ctx.set_tuning(a.vpt, a.G, a.tuned_ckpt, a.wpb)
        lib.idm_set_profiling(h, 1)
        mt = measure(a.tuned_steps, max(3, min(a.warmup, 3)), False)
        tuned = {"ckpt_interval": a.tuned_ckpt, "steps": a.tuned_steps,
                 "value": world * units_per_step * a.tuned_steps / (mt["ms"] * 1e-3),
                 "ms_per_step": mt["ms"] / a.tuned_steps,
                 "fwd_ms_per_timestep": mt["fwd_avg_ms"] / K, "bwd_ms_per_timestep": mt["bwd_avg_ms"] / K,
                 "roofline": adjoint_roofline(N, K, a.tuned_ckpt, mt["bwd_avg_ms"], n_sm, peaks, peak_kind),
                 "note": "the same workload with the checkpoint interval whose adjoint tape fits shared memory "
                         "(no tape blocks); checkpoints then take %.1f GB instead of %.2f GB"
                         % (16.0 * N * math.ceil(K / a.tuned_ckpt) / 1e9, 16.0 * N * math.ceil(K / a.ckpt) / 1e9)}
        ctx.set_tuning(a.vpt, a.G, a.ckpt, a.wpb)

    # ---- Sec. III-C events of the fitted and the true parameters ------------
    ctx.set_event_counting(True)
    ctx.event_counts()
    api.simulate(s_th, s_p, s_v, api.Scene(lane_off, s_len, a.per_lane), K, DT, A_MIN, ctx=ctx)
    ev_fit = ctx.event_counts()
    api.simulate(th_true, p_sorted, v_sorted, scene_sorted, K, DT, A_MIN, ctx=ctx)
    ev_true = ctx.event_counts()
    ctx.set_event_counting(False)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "vehicles_per_gpu": N, "lanes_per_gpu": L, "job_lanes": L_job,
                   "K": K, "iters_per_step": a.iters,
                   "ckpt_interval": a.ckpt, "vpt": a.vpt, "warps_per_segment": a.G, "warps_per_block": a.wpb,
                   "l2": "inputs larger than L2 (targets %.1f GB per GPU)" % (K * N * 4 / 1e9),
                   "parallelism": "dp%d (one scene sharded by lanes; FP64 loss-history all-reduce per step)" % world,
                   "fwd_ms_per_timestep": m["fwd_avg_ms"] / K, "bwd_ms_per_timestep": m["bwd_avg_ms"] / K,
                   "paper_context": "paper Fig. 1: < 30 ms per timestep forward and backward each at 2M vehicles "
                                    "(RTX A5000 or 16-thread Xeon W-2255), i.e. > 3.3e7 fwd+bwd vehicle-steps/s "
                                    "(a bound, not an exact figure: vs_baseline stays null)",
                   "final_mse_m2": final_loss},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": (ms_e2e / e2e_steps) if ms_e2e else None},
        "gpu_launches": launches_per_step * a.steps,
        "roofline": roofline,
        "clocks": m["clocks"],
        "events": {"fitted": ev_fit, "truth": ev_true,
                   "what": "vehicle-steps with the raw gap below the 0.1 m floor / within 0.5 m/s^2 of the kink of "
                           "max(-v/dt, a_min), over one simulation of the %d steps" % K},
    }
    net = None
    if world == 1 and not a.no_crossover:
        line["cpu_gpu_crossover"] = cpu_gpu_crossover(a, dev)
    if world == 1 and not a.no_recon:
        line["reconstruction"] = reconstruction(a, dev)
    if world == 1 and not a.no_pred:
        line["prediction"] = prediction(a, dev)
    if world == 1 and not a.no_batched:
        line["batched"] = batched(a, dev)
    if world == 1 and not a.no_init_experiment:
        line["time_to_fit"], net = time_to_fit(a, dev)
        if not a.no_long_horizon:
            line["long_horizon"] = long_horizon(a, dev, net)
        net.close()
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v1, secs1, desc = oracle_sample(iters=30)
        vc, secs_c, cores = oracle_all_cores(iters=10)
        line["cpu_baseline"] = {"value": vc, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d processes, each: %s" % (cores, desc.replace("30 fit", "10 fit")),
                                "seconds": secs_c,
                                "single_core": {"value": v1, "sample": desc, "seconds": secs1}}
    if tuned is not None:
        line["tuned_variant"] = tuned
    line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def summary(line):
    """The figures of every part of the metric in a few hundred characters,
    printed last so that the tail of the line carries them."""
    r = lambda x, n=4: (float("%.*g" % (n, x)) if isinstance(x, (int, float)) else x)
    out = {"fwd_bwd_vehicle_steps_per_s": r(line["value"]), "ckpt_interval": line["config"]["ckpt_interval"],
           "adjoint_ms": r(line["roofline"]["avg_launch_ms"]), "adjoint_fp32_frac": r(line["roofline"]["frac"], 3)}
    tv = line.get("tuned_variant")
    if tv:
        out["tuned_ckpt_%d" % tv["ckpt_interval"]] = {"value": r(tv["value"]),
                                                      "adjoint_ms": r(tv["roofline"]["avg_launch_ms"]),
                                                      "adjoint_fp32_frac": r(tv["roofline"]["frac"], 3)}
    ttf = line.get("time_to_fit")
    if ttf:
        f = ttf["fit"]
        last = str(max(int(k) for k in f["plain"]["rmse_m_at"]))
        out["time_to_fit_0.5m"] = {
            k: {"iterations": f[k]["iterations"], "s": r(f[k]["seconds"]) if f[k]["seconds"] else None,
                "rmse_m_last": r(f[k]["rmse_m_at"][last], 3)}
            for k in ("learned", "plain", "training_mean_ablation")}
        out["time_to_fit_0.5m"]["learned"]["init_ms"] = r(f["learned"]["init_ms"], 3)
        out["time_to_fit_0.5m"]["ms_per_iteration"] = r(f["ms_per_iteration"], 3)
    b = line.get("batched")
    if b:
        out["batched_vehicle_steps_per_s"] = r(b["vehicle_steps_per_s"])
    lh = line.get("long_horizon")
    if lh:
        out["long_horizon"] = {"rmse_fit_m": r(lh["rmse_fit_window_m"], 3), "rmse_pred_m": r(lh["rmse_prediction_m"], 3),
                               "fit_vehicle_steps_per_s": r(lh["fit_vehicle_steps_per_s"]),
                               "oracle_max_abs_diff_m": r(lh["oracle_check"]["max_abs_diff_m"], 3)}
    out["events_fitted"] = line["events"]["fitted"]
    return out


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank)
    return run_gpu(a, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
