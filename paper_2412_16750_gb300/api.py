"""PyTorch-facing API over libidm: device memory and streams come from torch,
every step of the simulation and its adjoint runs in libidm's kernels.

    ctx = Context()
    scene = Scene.from_lane_off(lane_off, length)            # CUDA tensors
    traj = IdmFunction.apply(theta, p_init, v_init, scene, K, dt)  # (K+1, N)
    traj.sum().backward()                                      # idm_backward

``theta`` is a (6, N) float32 tensor with rows (v0, T, s0, a_max, b, delta),
the paper's (v_targ, T_pref, s_min, a_max, a_pref, delta) of Eq. 1-2.
"""
from dataclasses import dataclass

import torch

from . import lib

PARAM_NAMES = ("v0", "T", "s0", "a_max", "b", "delta")


class Context:
    """Owns an idm_ctx_t (workspace on the current device)."""

    def __init__(self, workspace_cap_bytes=0, vpt=0, warps_per_segment=0, ckpt_interval=8, warps_per_block=8):
        self.handle = lib.idm_ctx_create(workspace_cap_bytes)
        self.set_tuning(vpt, warps_per_segment, ckpt_interval, warps_per_block)

    def set_tuning(self, vpt=0, warps_per_segment=0, ckpt_interval=8, warps_per_block=8):
        lib.idm_set_tuning(self.handle, vpt, warps_per_segment, ckpt_interval, warps_per_block)
        self.tuning = (vpt, warps_per_segment, ckpt_interval, warps_per_block)

    def set_fit_mode(self, mode):
        """How idm_fit runs its iterations: "auto", "graph" (one forward and
        one adjoint launch per iteration in a CUDA graph) or "single" (every
        iteration in one persistent launch); the results are identical."""
        code = {"auto": lib.IDM_FIT_AUTO, "graph": lib.IDM_FIT_GRAPH, "single": lib.IDM_FIT_SINGLE_LAUNCH}[mode]
        lib.idm_set_fit_mode(self.handle, code)
        self.fit_mode = mode

    def last_fit_form(self):
        """"graph" or "single" for the last fit on this context (None before one)."""
        return {lib.IDM_FIT_GRAPH: "graph", lib.IDM_FIT_SINGLE_LAUNCH: "single"}.get(
            lib.idm_last_fit_form(self.handle))

    def status(self, stream=None):
        rc, flags = lib.idm_status(self.handle, stream or torch.cuda.current_stream())
        return rc, flags

    def check_status(self):
        rc, flags = self.status()
        if rc != lib.IDM_OK:
            raise lib.IdmError(rc, lib.idm_last_error(self.handle))
        return flags

    def set_event_counting(self, on):
        """Count gap-floor hits and kink-band vehicle-steps in simulate /
        batch_forward (idm_set_event_counting)."""
        lib.idm_set_event_counting(self.handle, on)

    def event_counts(self, stream=None):
        """{"gap_floor_hits": n, "kink_near": n} since the last read (clears them)."""
        a, b = lib.idm_event_counts(self.handle, stream or torch.cuda.current_stream())
        return {"gap_floor_hits": a, "kink_near": b}

    def close(self):
        if self.handle is not None:
            lib.idm_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context():
    dev = torch.cuda.current_device()
    if dev not in _default_ctx:
        _default_ctx[dev] = Context()
    return _default_ctx[dev]


@dataclass
class Scene:
    lane_off: torch.Tensor  # int32 [L+1], CUDA
    length: torch.Tensor    # float32 [N], CUDA
    max_lane: int

    @staticmethod
    def from_lane_off(lane_off, length, max_lane=None):
        lane_off = lane_off.to(device="cuda", dtype=torch.int32).contiguous()
        length = length.to(device="cuda", dtype=torch.float32).contiguous()
        if max_lane is None:
            max_lane = int((lane_off[1:] - lane_off[:-1]).max().item()) if lane_off.numel() > 1 else 0
        return Scene(lane_off, length, max_lane)

    @property
    def n_vehicles(self):
        return self.length.numel()

    @property
    def n_lanes(self):
        return self.lane_off.numel() - 1

    def c(self):
        return lib.make_scene(self.lane_off, self.length, self.max_lane)


def _f32(t):
    return t.to(device="cuda", dtype=torch.float32).contiguous()


def _stream():
    return torch.cuda.current_stream()


def simulate(theta, p_init, v_init, scene, K, dt, a_min=-10.0, want_speed=False, ctx=None):
    """Positions (and speeds) over K steps, time-major (K+1, N)."""
    ctx = ctx or default_context()
    theta, p_init, v_init = _f32(theta), _f32(p_init), _f32(v_init)
    N = scene.n_vehicles
    traj = torch.empty((K + 1, N), device="cuda", dtype=torch.float32)
    vtraj = torch.empty((K + 1, N), device="cuda", dtype=torch.float32) if want_speed else None
    lib.idm_forward(ctx.handle, scene.c(), lib.make_params(theta), p_init, v_init, lib.make_sim(K, dt, a_min),
                    traj, vtraj, _stream())
    return (traj, vtraj) if want_speed else traj


def backward(theta, p_init, v_init, scene, K, dt, gP, gV=None, a_min=-10.0, ctx=None):
    """Adjoint from dense trajectory gradients: (g_theta (6,N), g_p_init, g_v_init)."""
    ctx = ctx or default_context()
    theta, p_init, v_init, gP = _f32(theta), _f32(p_init), _f32(v_init), _f32(gP)
    gV = _f32(gV) if gV is not None else None
    N = scene.n_vehicles
    g = torch.empty((6, N), device="cuda", dtype=torch.float32)
    gp = torch.empty(N, device="cuda", dtype=torch.float32)
    gv = torch.empty(N, device="cuda", dtype=torch.float32)
    lib.idm_backward(ctx.handle, scene.c(), lib.make_params(theta), p_init, v_init, lib.make_sim(K, dt, a_min),
                     gP, gV, lib.make_params(g), gp, gv, _stream())
    return g, gp, gv


def loss_grad(theta, p_init, v_init, scene, K, dt, targets, obs_stride=1, a_min=-10.0, ctx=None,
              want_state_grad=True):
    """Fused squared-error loss (sum over vehicles of each vehicle's mean)
    and its gradients: (loss float64 0-d tensor, g_theta, g_p_init, g_v_init)."""
    ctx = ctx or default_context()
    theta, p_init, v_init = _f32(theta), _f32(p_init), _f32(v_init)
    targets = _f32(targets) if targets is not None else None
    N = scene.n_vehicles
    loss = torch.zeros((), device="cuda", dtype=torch.float64)
    g = torch.empty((6, N), device="cuda", dtype=torch.float32)
    gp = torch.empty(N, device="cuda", dtype=torch.float32) if want_state_grad else None
    gv = torch.empty(N, device="cuda", dtype=torch.float32) if want_state_grad else None
    lib.idm_loss_grad(ctx.handle, scene.c(), lib.make_params(theta), p_init, v_init, lib.make_sim(K, dt, a_min),
                      targets, obs_stride, loss, lib.make_params(g), gp, gv, _stream())
    return loss, g, gp, gv


def fit(theta, p_init, v_init, scene, K, dt, targets, obs_stride, n_iter, lr0=0.1, lr1=0.01,
        box_lo=(20.0, 0.1, 1.0, 0.5, 0.1), box_hi=(60.0, 5.0, 10.0, 10.0, 5.0), a_min=-10.0, ctx=None,
        eval_targets=None):
    """Adam fit of (v0, T, s0, a_max, b) in place on a float32 (6, N) CUDA
    tensor; returns the float64 loss history (n_iter,).  With eval_targets
    (same layout as targets) returns (loss history, eval loss history): the
    second is the loss of every iterate against eval_targets."""
    ctx = ctx or default_context()
    assert theta.is_cuda and theta.dtype == torch.float32 and theta.is_contiguous()
    p_init, v_init, targets = _f32(p_init), _f32(v_init), _f32(targets)
    hist = torch.zeros(max(n_iter, 1), device="cuda", dtype=torch.float64)
    if eval_targets is None:
        lib.idm_fit(ctx.handle, scene.c(), lib.make_params(theta), p_init, v_init, lib.make_sim(K, dt, a_min),
                    targets, obs_stride, n_iter, lr0, lr1, box_lo, box_hi, hist, _stream())
        return hist[:n_iter]
    eval_targets = _f32(eval_targets)
    ehist = torch.zeros(max(n_iter, 1), device="cuda", dtype=torch.float64)
    lib.idm_fit_eval(ctx.handle, scene.c(), lib.make_params(theta), p_init, v_init, lib.make_sim(K, dt, a_min),
                     targets, obs_stride, n_iter, lr0, lr1, box_lo, box_hi, hist, eval_targets, ehist, _stream())
    return hist[:n_iter], ehist[:n_iter]


def layout(lane_id, pos, n_lanes, ctx=None):
    """Head-first lane order: (perm int32 [N], lane_off int32 [L+1], max_lane int32 [1])."""
    ctx = ctx or default_context()
    lane_id = lane_id.to(device="cuda", dtype=torch.int32).contiguous()
    pos = _f32(pos)
    N = lane_id.numel()
    perm = torch.empty(N, device="cuda", dtype=torch.int32)
    lane_off = torch.empty(n_lanes + 1, device="cuda", dtype=torch.int32)
    mx = torch.zeros(1, device="cuda", dtype=torch.int32)
    lib.idm_layout(ctx.handle, N, n_lanes, lane_id, pos, perm, lane_off, mx, _stream())
    return perm, lane_off, mx


def gather(perm, srcs, ctx=None):
    """[src[perm] for src in srcs] via idm_gather (float32 arrays)."""
    ctx = ctx or default_context()
    srcs = [_f32(s) for s in srcs]
    dsts = [torch.empty(perm.numel(), device="cuda", dtype=torch.float32) for _ in srcs]
    lib.idm_gather(ctx.handle, perm.numel(), perm, srcs, dsts, _stream())
    return dsts


class Batch:
    """Uneven scenarios for the idm_batch_* calls.  Host arrays (numpy or
    lists) describe the scenarios; the lane CSR and lengths are copied to the
    device once."""

    def __init__(self, scen_lane_off, K, dt, obs_stride, lane_off, length, a_min=-10.0):
        import numpy as np
        self.scen_lane_off = np.ascontiguousarray(scen_lane_off, dtype=np.int32)
        self.K = np.ascontiguousarray(K, dtype=np.int32)
        self.dt = np.ascontiguousarray(dt, dtype=np.float32)
        self.obs_stride = np.ascontiguousarray(obs_stride, dtype=np.int32)
        self.lane_off_host = np.ascontiguousarray(lane_off, dtype=np.int32)
        self.lane_off = torch.as_tensor(self.lane_off_host, device="cuda")
        self.length = _f32(torch.as_tensor(length))
        self.a_min = a_min
        self.n_scen = len(self.K)
        self.veh_off = self.lane_off_host[self.scen_lane_off]
        self.n_obs = self.K // self.obs_stride
        nv = np.diff(self.veh_off)
        self.traj_off = np.concatenate([[0], np.cumsum((self.K.astype(np.int64) + 1) * nv)])
        self.tgt_off = np.concatenate([[0], np.cumsum(self.n_obs.astype(np.int64) * nv)])

    def c(self):
        return lib.idm_batch_t(self.n_scen, self.scen_lane_off.ctypes.data, self.K.ctypes.data, self.dt.ctypes.data,
                               self.obs_stride.ctypes.data, self.a_min, len(self.lane_off_host) - 1,
                               int(self.lane_off_host[-1]), self.lane_off_host.ctypes.data, self.lane_off.data_ptr(),
                               self.length.data_ptr())

    @property
    def n_vehicles(self):
        return int(self.lane_off_host[-1])


def batch_forward(theta, p_init, v_init, batch, ctx=None):
    """Concatenated per-scenario trajectories (flat float32 tensor)."""
    ctx = ctx or default_context()
    traj = torch.empty(int(batch.traj_off[-1]), device="cuda", dtype=torch.float32)
    lib.idm_batch_forward(ctx.handle, batch.c(), lib.make_params(_f32(theta)), _f32(p_init), _f32(v_init), traj,
                          _stream())
    return traj


def batch_loss_grad(theta, p_init, v_init, batch, targets, ctx=None):
    """(per-scenario losses [S] float64, total, g_theta (6,N), g_p_init, g_v_init)."""
    ctx = ctx or default_context()
    N = batch.n_vehicles
    sl = torch.zeros(batch.n_scen, device="cuda", dtype=torch.float64)
    tot = torch.zeros((), device="cuda", dtype=torch.float64)
    g = torch.empty((6, N), device="cuda", dtype=torch.float32)
    gp = torch.empty(N, device="cuda", dtype=torch.float32)
    gv = torch.empty(N, device="cuda", dtype=torch.float32)
    lib.idm_batch_loss_grad(ctx.handle, batch.c(), lib.make_params(_f32(theta)), _f32(p_init), _f32(v_init),
                            _f32(targets), sl, tot, lib.make_params(g), gp, gv, _stream())
    return sl, tot, g, gp, gv


def batch_fit(theta, p_init, v_init, batch, targets, n_iter, lr0=0.1, lr1=0.01, box_lo=(20.0, 0.1, 1.0, 0.5, 0.1),
              box_hi=(60.0, 5.0, 10.0, 10.0, 5.0), ctx=None):
    """In-place Adam fit over a batch; returns (loss history (n_iter,), per-scenario losses of the last iteration)."""
    ctx = ctx or default_context()
    assert theta.is_cuda and theta.dtype == torch.float32 and theta.is_contiguous()
    hist = torch.zeros(max(n_iter, 1), device="cuda", dtype=torch.float64)
    sl = torch.zeros(batch.n_scen, device="cuda", dtype=torch.float64)
    lib.idm_batch_fit(ctx.handle, batch.c(), lib.make_params(theta), _f32(p_init), _f32(v_init), _f32(targets), n_iter,
                      lr0, lr1, box_lo, box_hi, hist, sl, _stream())
    return hist[:n_iter], sl


class IdmFunction(torch.autograd.Function):
    """Differentiable simulation: forward = idm_forward, backward = idm_backward."""

    @staticmethod
    def forward(fctx, theta, p_init, v_init, scene, K, dt, a_min=-10.0, ctx=None):
        ctx = ctx or default_context()
        traj = simulate(theta, p_init, v_init, scene, K, dt, a_min, ctx=ctx)
        fctx.save_for_backward(theta, p_init, v_init)
        fctx.cfg = (scene, K, dt, a_min, ctx)
        return traj

    @staticmethod
    def backward(fctx, gtraj):
        theta, p_init, v_init = fctx.saved_tensors
        scene, K, dt, a_min, ctx = fctx.cfg
        g, gp, gv = backward(theta, p_init, v_init, scene, K, dt, gtraj.contiguous(), None, a_min, ctx=ctx)
        return g, gp, gv, None, None, None, None, None


# ---------------------------------------------------------------------------
# Learned initializer (include/idm_mlp.h; no counterpart in the paper)
# ---------------------------------------------------------------------------

BOX_LO = (20.0, 0.1, 1.0, 0.5, 0.1)
BOX_HI = (60.0, 5.0, 10.0, 10.0, 5.0)


class Mlp:
    """The 80-256-256-256-5 GELU network of the learned initializer: bf16
    weights on the tensor cores, FP32 master weights and Adam state."""

    def __init__(self, max_batch=8192, weights=None):
        self.handle = lib.idm_mlp_create(max_batch)
        self.max_batch = max_batch
        if weights is not None:
            self.set_weights(weights)

    def set_weights(self, w):
        w = torch.as_tensor(w).to(device="cuda", dtype=torch.float32).contiguous()
        assert w.numel() == lib.IDM_MLP_N_PARAMS
        lib.idm_mlp_set_weights(self.handle, w, _stream())
        torch.cuda.current_stream().synchronize()  # the copy source may be a temporary

    def get_weights(self):
        w = torch.empty(lib.IDM_MLP_N_PARAMS, device="cuda", dtype=torch.float32)
        lib.idm_mlp_get_weights(self.handle, w, _stream())
        return w

    def forward(self, X):
        """sigmoid outputs (B, 5) of bf16 features X (B, 80)."""
        B = X.shape[0]
        out = torch.empty((B, 5), device="cuda", dtype=torch.float32)
        lib.idm_mlp_forward(self.handle, _bf16(X), B, out, _stream())
        return out

    def predict_params(self, X, theta, box_lo=BOX_LO, box_hi=BOX_HI):
        """Writes rows 0-4 (v0, T, s0, a_max, b) of the (6, B) tensor theta."""
        assert theta.is_cuda and theta.dtype == torch.float32 and theta.is_contiguous()
        B = X.shape[0]
        lib.idm_mlp_predict_params(self.handle, _bf16(X), B, lib.make_params(theta), box_lo, box_hi, _stream())
        return theta

    def loss_grad(self, X, labels):
        B = X.shape[0]
        loss = torch.zeros((), device="cuda", dtype=torch.float64)
        grad = torch.empty(lib.IDM_MLP_N_PARAMS, device="cuda", dtype=torch.float32)
        lib.idm_mlp_loss_grad(self.handle, _bf16(X), _f32(labels), B, loss, grad, _stream())
        return loss, grad

    def train_step(self, X, labels, lr):
        loss = torch.zeros((), device="cuda", dtype=torch.float64)
        lib.idm_mlp_train_step(self.handle, _bf16(X), _f32(labels), X.shape[0], lr, loss, _stream())
        return loss

    def train(self, X, labels, batch, n_steps, lr0=1e-3, lr1=1e-4):
        """n_steps Adam steps over consecutive batches of (X, labels); returns
        the loss history (float64, n_steps)."""
        hist = torch.zeros(max(n_steps, 1), device="cuda", dtype=torch.float64)
        lib.idm_mlp_train(self.handle, _bf16(X), _f32(labels), X.shape[0], batch, n_steps, lr0, lr1, hist,
                          _stream())
        return hist[:n_steps]

    def status(self):
        return lib.idm_mlp_status(self.handle, _stream())

    def clear_status(self):
        lib.idm_mlp_clear_status(self.handle, _stream())

    def set_wait_limit(self, polls):
        """Polls per tensor-core wait before a kernel gives up (0 = default)."""
        lib.idm_mlp_set_wait_limit(self.handle, polls)

    def close(self):
        if self.handle is not None:
            lib.idm_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bf16(t):
    assert t.is_cuda and t.dtype == torch.bfloat16 and t.is_contiguous()
    return t


def mlp_features(scene, p_init, v_init, K, dt, targets, obs_stride=1, perm=None, theta=None, box_lo=BOX_LO,
                 box_hi=BOX_HI):
    """Feature rows (bf16 (n, 80)) of the vehicles perm (default all); with
    theta (6, N) also the normalized labels (n, 5)."""
    p_init, v_init, targets = _f32(p_init), _f32(v_init), _f32(targets)
    perm_t = perm.to(device="cuda", dtype=torch.int32).contiguous() if perm is not None else None
    n = perm_t.numel() if perm_t is not None else scene.n_vehicles
    X = torch.empty((n, lib.IDM_MLP_IN), device="cuda", dtype=torch.bfloat16)
    labels = None
    if theta is not None:
        labels = torch.empty((n, 5), device="cuda", dtype=torch.float32)
    lib.idm_mlp_features(scene.c(), p_init, v_init, lib.make_sim(K, dt, -10.0), targets, obs_stride, perm_t, n, X,
                         lib.make_params(theta) if theta is not None else None, labels, box_lo, box_hi, _stream())
    return (X, labels) if theta is not None else X


# ---- single-trajectory filtering / reconstruction mode (Sec. IV-A) ----------

# Sec. IV-A: the five parameters start at v_targ 50, T_pref 1, s_min 5,
# a_max 10, a_pref 2 (delta 4, not fitted) inside the boxes below; the
# virtual leader starts at a 10 m gap and zero speed difference.
RECON_INIT = (50.0, 1.0, 5.0, 10.0, 2.0, 4.0)
RECON_BOX_LO = (20.0, 0.1, 1.0, 5.0, 0.1)
RECON_BOX_HI = (60.0, 5.0, 10.0, 10.0, 5.0)
RECON_DP0 = 10.0
RECON_DV0 = 0.0


class Recon:
    """Observed trajectories (CSR over trajectories) prepared for the
    reconstruction mode: nearest steps, horizons K and initial states come
    from idm_recon_prepare.  Per-step arrays are time-major with k_max rows
    and a row stride ld = N rounded up to 32 (so that rows can be staged
    with 16-byte copies); the methods accept (k_max, N) or (k_max, ld)
    tensors and return (.., N) views."""

    def __init__(self, obs_off, obs_t, obs_p, dt, a_min=-10.0, ctx=None, ld=None):
        self.ctx = ctx or default_context()
        self.obs_off = obs_off.to(device="cuda", dtype=torch.int32).contiguous()
        self.obs_t = _f32(obs_t)
        self.obs_p = _f32(obs_p)
        self.N = self.obs_off.numel() - 1
        self.n_obs = self.obs_p.numel()
        self.dt, self.a_min = float(dt), float(a_min)
        self.obs_k = torch.empty(max(self.n_obs, 1), device="cuda", dtype=torch.int32)
        self.K = torch.empty(max(self.N, 1), device="cuda", dtype=torch.int32)
        self.p_init = torch.empty(max(self.N, 1), device="cuda", dtype=torch.float32)
        self.v_init = torch.empty(max(self.N, 1), device="cuda", dtype=torch.float32)
        km = lib.idm_recon_prepare(self.ctx.handle, self.N, self.n_obs, self.obs_off, self.obs_t, self.obs_p,
                                   self.dt, self.obs_k, self.K, self.p_init, self.v_init, True, _stream())
        self.k_max = max(int(km), 1)
        self.ld = ld if ld is not None else max(32, -(-self.N // 32) * 32)
        assert self.ld >= self.N

    def c(self):
        return lib.idm_recon_t(self.N, self.k_max, self.ld, self.n_obs, lib.ptr(self.obs_off).value,
                               lib.ptr(self.obs_t).value, lib.ptr(self.obs_p).value, lib.ptr(self.obs_k).value,
                               lib.ptr(self.K).value, lib.ptr(self.p_init).value, lib.ptr(self.v_init).value,
                               self.dt, self.a_min)

    def _rows(self, x):
        """A (k_max, N) or (k_max, ld) per-step tensor as (k_max, ld) float32 contiguous."""
        x = _f32(x)
        assert x.shape[0] == self.k_max, "per-step arrays need k_max rows"
        if x.shape[1] == self.ld:
            return x
        y = torch.zeros((self.k_max, self.ld), device="cuda", dtype=torch.float32)
        y[:, :x.shape[1]] = x
        return y

    def init_vars(self):
        """(theta (6, N), dp, dv (k_max, ld)) at the paper's starting point."""
        theta = torch.tensor(RECON_INIT, dtype=torch.float32, device="cuda")[:, None].repeat(1, self.N).contiguous()
        dp = torch.full((self.k_max, self.ld), RECON_DP0, device="cuda", dtype=torch.float32)
        dv = torch.full((self.k_max, self.ld), RECON_DV0, device="cuda", dtype=torch.float32)
        return theta, dp, dv

    def forward(self, theta, dp, dv):
        """(P, V (k_max+1, N), A (k_max, N))."""
        theta, dp, dv = _f32(theta), self._rows(dp), self._rows(dv)
        P = torch.empty((self.k_max + 1, self.ld), device="cuda", dtype=torch.float32)
        V = torch.empty_like(P)
        A = torch.empty((self.k_max, self.ld), device="cuda", dtype=torch.float32)
        lib.idm_recon_forward(self.ctx.handle, self.c(), lib.make_params(theta), dp, dv, P, V, A, _stream())
        n = self.N
        return P[:, :n], V[:, :n], A[:, :n]

    def loss_grad(self, theta, dp, dv):
        """(loss float64 0-d, g_theta (6, N), g_dp, g_dv (k_max, N), g_p_init, g_v_init)."""
        theta, dp, dv = _f32(theta), self._rows(dp), self._rows(dv)
        loss = torch.zeros((), device="cuda", dtype=torch.float64)
        g = torch.empty((6, max(self.N, 1)), device="cuda", dtype=torch.float32)
        gdp = torch.empty((self.k_max, self.ld), device="cuda", dtype=torch.float32)
        gdv = torch.empty_like(gdp)
        gp = torch.empty(max(self.N, 1), device="cuda", dtype=torch.float32)
        gv = torch.empty(max(self.N, 1), device="cuda", dtype=torch.float32)
        lib.idm_recon_loss_grad(self.ctx.handle, self.c(), lib.make_params(theta), dp, dv, loss,
                                lib.make_params(g), gdp, gdv, gp, gv, _stream())
        n = self.N
        return loss, g[:, :n], gdp[:, :n], gdv[:, :n], gp[:n], gv[:n]

    def fit(self, theta, dp, dv, n_iter=500, lr0=0.1, lr1=0.01, box_lo=RECON_BOX_LO, box_hi=RECON_BOX_HI):
        """Adam fit in place on theta (6, N) and dp, dv ((k_max, N) or
        (k_max, ld)), float32 CUDA contiguous; returns the float64 loss
        history (n_iter,)."""
        for t in (theta, dp, dv):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        dpw, dvw = self._rows(dp), self._rows(dv)
        hist = torch.zeros(max(n_iter, 1), device="cuda", dtype=torch.float64)
        lib.idm_recon_fit(self.ctx.handle, self.c(), lib.make_params(theta), dpw, dvw, n_iter, lr0, lr1, box_lo,
                          box_hi, hist, _stream())
        if dpw.data_ptr() != dp.data_ptr():
            dp.copy_(dpw[:, :dp.shape[1]])
        if dvw.data_ptr() != dv.data_ptr():
            dv.copy_(dvw[:, :dv.shape[1]])
        return hist[:n_iter]

    def metrics(self, theta, dp, dv):
        """float64 (4,): Pos. (fraction), mean |a*|, std |a*|, Imp. (fraction)."""
        theta, dp, dv = _f32(theta), self._rows(dp), self._rows(dv)
        out = torch.zeros(4, device="cuda", dtype=torch.float64)
        lib.idm_recon_metrics(self.ctx.handle, self.c(), lib.make_params(theta), dp, dv, out, _stream())
        return out


# ---- lane geometry and training-free prediction (Sec. IV-B, Sec. V-C) -------

PRED_LENGTH = 4.5          # vehicle length (m) used for the gaps of projected agents
# the fitting box of the lane fit (a_max down to 0.5 m/s^2), from the start RECON_INIT
PRED_BOX_LO = (20.0, 0.1, 1.0, 0.5, 0.1)
PRED_BOX_HI = (60.0, 5.0, 10.0, 10.0, 5.0)


class Lanes:
    """Lane centre lines (polyline CSR) on the device, with their cumulative
    arc lengths from idm_lane_prepare."""

    def __init__(self, pt_off, px, py, ctx=None):
        self.ctx = ctx or default_context()
        self.pt_off = pt_off.to(device="cuda", dtype=torch.int32).contiguous()
        self.px, self.py = _f32(px), _f32(py)
        self.n_lanes = self.pt_off.numel() - 1
        self.n_points = self.px.numel()
        self.lane_len = torch.empty(self.n_points, device="cuda", dtype=torch.float32)
        lib.idm_lane_prepare(self.ctx.handle, self.n_lanes, self.n_points, self.pt_off, self.px, self.py,
                             self.lane_len, _stream())

    def c(self):
        return lib.idm_lanes_t(self.n_lanes, self.n_points, self.pt_off.data_ptr(), self.px.data_ptr(),
                               self.py.data_ptr(), self.lane_len.data_ptr())

    def project(self, x, y, lane_lo, lane_hi=None, want=("lane", "s", "d")):
        """Points (x, y) of shape (rows, cols) onto lanes: (lane, s, d) of the same shape."""
        x, y = _f32(x), _f32(y)
        rows, cols = (1, x.numel()) if x.dim() == 1 else tuple(x.shape)
        lane = torch.empty((rows, cols), device="cuda", dtype=torch.int32) if "lane" in want else None
        s = torch.empty((rows, cols), device="cuda", dtype=torch.float32) if "s" in want else None
        d = torch.empty((rows, cols), device="cuda", dtype=torch.float32) if "d" in want else None
        lo = lane_lo.to(device="cuda", dtype=torch.int32).contiguous()
        hi = lane_hi.to(device="cuda", dtype=torch.int32).contiguous() if lane_hi is not None else None
        lib.idm_lane_project(self.ctx.handle, self.c(), rows, cols, x, y, lo, hi, lane, s, d, _stream())
        return lane, s, d

    def unproject(self, s, lane_of_col):
        s = _f32(s)
        rows, cols = (1, s.numel()) if s.dim() == 1 else tuple(s.shape)
        x = torch.empty((rows, cols), device="cuda", dtype=torch.float32)
        y = torch.empty_like(x)
        lib.idm_lane_unproject(self.ctx.handle, self.c(), rows, cols, s,
                               lane_of_col.to(device="cuda", dtype=torch.int32).contiguous(), x, y, _stream())
        return x, y


def rollout_state(s_rows, row_a, row_b, dt, ctx=None):
    ctx = ctx or default_context()
    s_rows = _f32(s_rows)
    N = s_rows.shape[1]
    p = torch.empty(N, device="cuda", dtype=torch.float32)
    v = torch.empty(N, device="cuda", dtype=torch.float32)
    lib.idm_rollout_state(ctx.handle, N, s_rows, row_a, row_b, dt, p, v, _stream())
    return p, v


def displacement(px, py, tx, ty, miss_m=2.0, ctx=None):
    """(ade [N], fde [N], sums float64 [3]) of time-major (F, N) predictions."""
    ctx = ctx or default_context()
    F, N = px.shape
    ade = torch.empty(N, device="cuda", dtype=torch.float32)
    fde = torch.empty(N, device="cuda", dtype=torch.float32)
    sums = torch.zeros(3, device="cuda", dtype=torch.float64)
    lib.idm_displacement(ctx.handle, F, N, _f32(px), _f32(py), _f32(tx), _f32(ty), miss_m, ade, fde, sums,
                         _stream())
    return ade, fde, sums


def predict_rollout(lanes, x_hist, y_hist, lane_lo, lane_hi, dt, n_fut, n_iter=500, lr0=0.1, lr1=0.01,
                    box_lo=PRED_BOX_LO, box_hi=PRED_BOX_HI, theta0=RECON_INIT, a_min=-10.0, ctx=None, tune=False):
    """Training-free prediction (Sec. IV-B, V-C): assign every agent to the
    nearest candidate lane at the last history frame, project its history
    onto that lane, order the agents lane by lane (head first), fit the IDM
    parameters to the H - 1 history steps, roll out n_fut steps from the last
    history frame and project the rollout back onto the lane centre lines.
    x_hist, y_hist: (H, N).  Returns a dict (agents in the fitted order given
    by perm): perm, lane, theta, loss history, s_hist (H, N), x, y (n_fut, N).
    tune: pick the fit's kernel shape with the autotuner (cached per GPU and
    problem signature) before fitting."""
    ctx = ctx or default_context()
    st = _stream()
    x_hist, y_hist = _f32(x_hist), _f32(y_hist)
    H, N = x_hist.shape
    lane, _, _ = lanes.project(x_hist[H - 1], y_hist[H - 1], lane_lo, lane_hi, want=("lane",))
    lane = lane.view(N)
    _, s_hist, _ = lanes.project(x_hist, y_hist, lane, None, want=("s",))
    perm, lane_off, _ = layout(lane, s_hist[0], lanes.n_lanes, ctx=ctx)
    s_sorted = torch.empty_like(s_hist)
    lib.idm_gather_rows(ctx.handle, N, H, perm, s_hist, s_sorted, st)
    lane_sorted = torch.empty(N, device="cuda", dtype=torch.int32)
    lib.idm_gather(ctx.handle, N, perm, [lane.view(torch.float32)], [lane_sorted.view(torch.float32)], st)
    scene = Scene.from_lane_off(lane_off, torch.full((N,), PRED_LENGTH, device="cuda", dtype=torch.float32))
    p0, v0 = rollout_state(s_sorted, 0, 1, dt, ctx=ctx)
    theta = torch.tensor(theta0, dtype=torch.float32, device="cuda")[:, None].repeat(1, N).contiguous()
    if tune:
        # time what runs: a short fit (the shape decides its form and tape
        # depth as well as the per-step cost), on a scratch copy
        from . import tune as _tune
        sig = _tune.signature(scene.max_lane, N, H - 1, 1, kind="predict-fit")
        scratch = theta.clone()
        _tune.tuned(ctx, lambda c: fit(scratch, p0, v0, scene, H - 1, dt, s_sorted[1:], 1, 20, lr0, lr1, box_lo,
                                       box_hi, a_min, ctx=c), scene.max_lane, sig)
    hist = fit(theta, p0, v0, scene, H - 1, dt, s_sorted[1:], 1, n_iter, lr0, lr1, box_lo, box_hi, a_min, ctx=ctx)
    pr, vr = rollout_state(s_sorted, H - 2, H - 1, dt, ctx=ctx)
    traj = simulate(theta, pr, vr, scene, n_fut, dt, a_min, ctx=ctx)
    x, y = lanes.unproject(traj[1:], lane_sorted)
    return dict(perm=perm, lane=lane_sorted, lane_off=lane_off, theta=theta, loss=hist, s_hist=s_sorted, x=x, y=y,
                p_roll=pr, v_roll=vr)
