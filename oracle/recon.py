"""ctypes front end of the FP64 single-trajectory reconstruction oracle
(``recon_oracle.c``, paper Sec. IV-A): one ego vehicle per trajectory behind
a virtual leader whose gap dp_k and speed difference dv_k are free variables.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Observations are a
CSR: trajectory i owns obs_off[i] .. obs_off[i+1]-1 (time order) with
timestamps obs_t (s, from the trajectory's start), nearest steps obs_k and
positions obs_p.  dp, dv are time-major (K_max, N); P, V (K_max+1, N).
"""
import ctypes

import numpy as np

from .ref import _f64, _i32, _load, _p, _pi, _rows


def nearest_step(t, dt):
    return _load().orc_recon_nearest_step(float(t), float(dt))


def nearest_steps(t, dt):
    """Nearest step of every timestamp (int32 array)."""
    t = _f64(t)
    k = np.empty(len(t), dtype=np.int32)
    _load().orc_recon_nearest_steps(ctypes.c_int64(len(t)), _p(t), ctypes.c_double(dt), _pi(k))
    return k


def horizons(obs_off, obs_k):
    """K[i] = the nearest step of trajectory i's last observation (0 if none)."""
    obs_off = np.asarray(obs_off)
    n = np.diff(obs_off)
    last = np.maximum(obs_off[1:] - 1, 0)
    return np.where(n > 0, np.asarray(obs_k)[last] if len(obs_k) else 0, 0).astype(np.int32)


def init_state(obs_off, obs_t, obs_p):
    lib = _load()
    obs_off = _i32(obs_off)
    N = len(obs_off) - 1
    p0, v0 = np.empty(N), np.empty(N)
    lib.orc_recon_init_state(ctypes.c_int(N), _pi(obs_off), _p(_f64(obs_t)), _p(_f64(obs_p)), _p(p0), _p(v0))
    return p0, v0


def forward(K, dp, dv, theta, p0, v0, dt, a_min=-10.0):
    """(P, V, A) of all trajectories."""
    lib = _load()
    K = _i32(K)
    N = len(K)
    dp, dv = _f64(dp).reshape(-1, N), _f64(dv).reshape(-1, N)
    K_max = dp.shape[0]
    th = _f64(theta).reshape(6, N)
    P, V, A = np.empty((K_max + 1, N)), np.empty((K_max + 1, N)), np.empty((max(K_max, 1), N))
    lib.orc_recon_forward(ctypes.c_int(N), ctypes.c_int(K_max), _pi(K), _p(dp), _p(dv), _rows(th), _p(_f64(p0)),
                          _p(_f64(v0)), ctypes.c_double(dt), ctypes.c_double(a_min), _p(P), _p(V), _p(A))
    return P, V, A[:K_max]


def mae_seed(K, obs_off, obs_k, obs_p, P):
    """(L, gP) of the summed absolute error."""
    lib = _load()
    K = _i32(K)
    N = len(K)
    P = _f64(P)
    K_max = P.shape[0] - 1
    gP = np.zeros_like(P)
    L = lib.orc_recon_mae_seed(ctypes.c_int(N), ctypes.c_int(K_max), _pi(K), _pi(_i32(obs_off)), _pi(_i32(obs_k)),
                               _p(_f64(obs_p)), _p(P), _p(gP))
    return L, gP


def adjoint(K, dp, dv, theta, dt, V, gP, a_min=-10.0):
    """(g_theta (6, N), g_dp, g_dv (K_max, N), g_p0, g_v0)."""
    lib = _load()
    K = _i32(K)
    N = len(K)
    dp, dv = _f64(dp).reshape(-1, N), _f64(dv).reshape(-1, N)
    K_max = dp.shape[0]
    th = _f64(theta).reshape(6, N)
    g = np.zeros((6, N))
    gdp, gdv = np.zeros((max(K_max, 1), N)), np.zeros((max(K_max, 1), N))
    gp0, gv0 = np.zeros(N), np.zeros(N)
    lib.orc_recon_adjoint(ctypes.c_int(N), ctypes.c_int(K_max), _pi(K), _p(dp), _p(dv), _rows(th), ctypes.c_double(dt),
                          ctypes.c_double(a_min), _p(_f64(V)), _p(_f64(gP)), _rows(g), _p(gdp), _p(gdv), _p(gp0),
                          _p(gv0))
    return g, gdp[:K_max], gdv[:K_max], gp0, gv0


def fit(K, dp, dv, theta, p0, v0, dt, obs_off, obs_k, obs_p, n_iter, lr0, lr1, lo, hi, a_min=-10.0):
    """Adam fit; returns (theta, dp, dv, loss history)."""
    lib = _load()
    K = _i32(K)
    N = len(K)
    dp, dv = _f64(dp).reshape(-1, N).copy(), _f64(dv).reshape(-1, N).copy()
    K_max = dp.shape[0]
    th = _f64(theta).reshape(6, N).copy()
    hist = np.empty(max(n_iter, 1))
    lib.orc_recon_fit(ctypes.c_int(N), ctypes.c_int(K_max), _pi(K), _p(dp), _p(dv), _rows(th), _p(_f64(p0)),
                      _p(_f64(v0)), ctypes.c_double(dt), ctypes.c_double(a_min), _pi(_i32(obs_off)),
                      _pi(_i32(obs_k)), _p(_f64(obs_p)), ctypes.c_int(n_iter), ctypes.c_double(lr0),
                      ctypes.c_double(lr1), _p(_f64(lo)), _p(_f64(hi)), _p(hist))
    return th, dp, dv, hist[:n_iter]


def metrics(K, obs_off, obs_k, obs_p, P, A):
    """(Pos., mean |a|, std |a|, Imp.)."""
    lib = _load()
    K = _i32(K)
    N = len(K)
    out = np.zeros(4)
    P, A = _f64(P), _f64(A)
    K_max = P.shape[0] - 1
    lib.orc_recon_metrics(ctypes.c_int(N), ctypes.c_int(K_max), _pi(K), _pi(_i32(obs_off)), _pi(_i32(obs_k)),
                          _p(_f64(obs_p)), _p(P), _p(A if A.size else np.zeros((1, N))), _p(out))
    return tuple(out)
