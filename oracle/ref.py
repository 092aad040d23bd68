"""ctypes front end of the FP64 C oracle (``idm_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function takes
and returns float64 numpy arrays; parameters travel as a (6, N) array in the
order ``PARAM_NAMES`` (v0, T, s0, a_max, b, delta), the paper's
(v_targ, T_pref, s_min, a_max, a_pref, delta) of Eq. 1-2.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

PARAM_NAMES = ("v0", "T", "s0", "a_max", "b", "delta")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "idm_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "recon_oracle.c"))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def build(force=False):
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp] + list(_SRCS) + ["-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_forward.restype = None
            lib.orc_mse_seed.restype = ctypes.c_double
            lib.orc_adjoint.restype = None
            lib.orc_adam_step.restype = None
            lib.orc_lr.restype = ctypes.c_double
            lib.orc_lr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.orc_fit.restype = None
            lib.orc_layout.restype = ctypes.c_int
            lib.orc_recon_nearest_step.restype = ctypes.c_int
            lib.orc_recon_nearest_step.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_recon_mae_seed.restype = ctypes.c_double
            for name in ("orc_recon_init_state", "orc_recon_forward", "orc_recon_adjoint", "orc_recon_fit",
                         "orc_recon_metrics", "orc_recon_nearest_steps"):
                getattr(lib, name).restype = None
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(_dp)


def _pi(a):
    return a.ctypes.data_as(_ip)


def _rows(arr2d):
    """(6, N) contiguous array -> ctypes array of 6 row pointers."""
    rows = (_dp * arr2d.shape[0])()
    for q in range(arr2d.shape[0]):
        rows[q] = arr2d[q].ctypes.data_as(_dp)
    return rows


def forward(lane_off, length, theta, p_init, v_init, K, dt, a_min=-10.0, want_accel=False):
    """Simulate K steps. Returns (P, V) of shape (K+1, N) [, A of shape (K, N)]."""
    lib = _load()
    lane_off = _i32(lane_off)
    N = int(lane_off[-1])
    theta = _f64(theta).reshape(6, N)
    length, p_init, v_init = _f64(length), _f64(p_init), _f64(v_init)
    P = np.empty((K + 1, N))
    V = np.empty((K + 1, N))
    A = np.empty((max(K, 0), N)) if want_accel else None
    lib.orc_forward(ctypes.c_int(len(lane_off) - 1), _pi(lane_off), _p(length), _rows(theta),
                    _p(p_init), _p(v_init), ctypes.c_int(K), ctypes.c_double(dt),
                    ctypes.c_double(a_min), _p(P), _p(V), _p(A) if A is not None else None)
    return (P, V, A) if want_accel else (P, V)


def mse_seed(P, targets, obs_stride):
    """Loss sum_i mean_j (P[j s, i] - y[j-1, i])^2 and its seed dL/dP."""
    lib = _load()
    P = _f64(P)
    K = P.shape[0] - 1
    N = P.shape[1]
    n_obs = K // obs_stride
    targets = _f64(targets).reshape(n_obs, N) if n_obs > 0 else np.zeros((1, N))
    gP = np.empty_like(P)
    L = lib.orc_mse_seed(ctypes.c_int(N), ctypes.c_int(K), _p(P), _p(targets),
                         ctypes.c_int(obs_stride), _p(gP))
    return L, gP


def adjoint(lane_off, length, theta, K, dt, P, V, gP, gV=None, a_min=-10.0):
    """Reverse-time adjoint. Returns (g_theta (6, N), g_p_init, g_v_init)."""
    lib = _load()
    lane_off = _i32(lane_off)
    N = int(lane_off[-1])
    theta = _f64(theta).reshape(6, N)
    length, P, V, gP = _f64(length), _f64(P), _f64(V), _f64(gP)
    gV = _f64(gV) if gV is not None else None
    gth = np.empty((6, N))
    gp0 = np.empty(N)
    gv0 = np.empty(N)
    lib.orc_adjoint(ctypes.c_int(len(lane_off) - 1), _pi(lane_off), _p(length), _rows(theta),
                    ctypes.c_int(K), ctypes.c_double(dt), ctypes.c_double(a_min),
                    _p(P), _p(V), _p(gP), _p(gV) if gV is not None else None,
                    _rows(gth), _p(gp0), _p(gv0))
    return gth, gp0, gv0


def adam_step(theta5, g5, m5, v5, t, lr, lo, hi, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam + box projection on (5, N) arrays (all float64, contiguous)."""
    lib = _load()
    for a in (theta5, m5, v5):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g5 = _f64(g5)
    lo, hi = _f64(lo), _f64(hi)
    lib.orc_adam_step(ctypes.c_int(theta5.shape[1]), _rows(theta5), _rows(g5), _rows(m5), _rows(v5),
                      ctypes.c_int(t), ctypes.c_double(lr), ctypes.c_double(beta1),
                      ctypes.c_double(beta2), ctypes.c_double(eps), _p(lo), _p(hi))


def lr_schedule(it, n_iter, lr0, lr1):
    return _load().orc_lr(it, n_iter, lr0, lr1)


def fit(lane_off, length, theta, p_init, v_init, K, dt, targets, obs_stride, n_iter,
        lr0, lr1, lo, hi, a_min=-10.0):
    """Adam fit; returns (theta_fitted (6, N), loss_hist (n_iter,))."""
    lib = _load()
    lane_off = _i32(lane_off)
    N = int(lane_off[-1])
    th = _f64(theta).reshape(6, N).copy()
    n_obs = K // obs_stride
    targets = _f64(targets).reshape(max(n_obs, 1), N)
    hist = np.empty(n_iter)
    lo, hi = _f64(lo), _f64(hi)
    lib.orc_fit(ctypes.c_int(len(lane_off) - 1), _pi(lane_off), _p(_f64(length)), _rows(th),
                _p(_f64(p_init)), _p(_f64(v_init)), ctypes.c_int(K), ctypes.c_double(dt),
                ctypes.c_double(a_min), _p(targets), ctypes.c_int(obs_stride), ctypes.c_int(n_iter),
                ctypes.c_double(lr0), ctypes.c_double(lr1), _p(lo), _p(hi), _p(hist))
    return th, hist


def layout(lane_id, pos, n_lanes):
    """Sort by (lane asc, position desc, index asc). Returns (perm, lane_off)."""
    lib = _load()
    lane_id = _i32(lane_id)
    pos = _f64(pos)
    N = lane_id.shape[0]
    perm = np.empty(N, dtype=np.int32)
    lane_off = np.empty(n_lanes + 1, dtype=np.int32)
    rc = lib.orc_layout(ctypes.c_int(N), ctypes.c_int(n_lanes), _pi(lane_id), _p(pos), _pi(perm), _pi(lane_off))
    if rc != 0:
        raise ValueError("lane id out of range")
    return perm, lane_off
