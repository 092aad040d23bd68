"""ctypes binding of libidm_cpu (include/idm_cpu.h), the multi-threaded CPU
backend: same names, argument marshalling only, numpy host arrays.

An explicit backend the caller chooses; the CUDA API (``lib``/``api``) never
falls back to it.  Raises ``RuntimeError`` when the library is not built.
"""
import ctypes
import os

import numpy as np

from .lib import IDM_OK, idm_params_t, idm_sim_t

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libidm_cpu.so")

_vp = ctypes.c_void_p


class idm_cpu_scene_t(ctypes.Structure):
    _fields_ = [("n_lanes", ctypes.c_int32), ("n_vehicles", ctypes.c_int32), ("lane_off", _vp), ("length", _vp)]


_SIGS = {
    "idm_cpu_max_threads": (ctypes.c_int, []),
    "idm_cpu_forward": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(idm_cpu_scene_t), ctypes.POINTER(idm_params_t),
                                       _vp, _vp, ctypes.POINTER(idm_sim_t), _vp, _vp]),
    "idm_cpu_loss_grad": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(idm_cpu_scene_t),
                                         ctypes.POINTER(idm_params_t), _vp, _vp, ctypes.POINTER(idm_sim_t), _vp,
                                         ctypes.c_int32, _vp, ctypes.POINTER(idm_params_t), _vp, _vp]),
    "idm_cpu_fit": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(idm_cpu_scene_t), ctypes.POINTER(idm_params_t), _vp,
                                   _vp, ctypes.POINTER(idm_sim_t), _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                   ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                   _vp]),
}

_lib = None


def exported_symbols():
    return sorted(_SIGS)


def load(path=None):
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libidm_cpu.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class CpuError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("libidm_cpu error %d in %s" % (code, what))
        self.code = code


def _check(rc, what):
    if rc != IDM_OK:
        raise CpuError(rc, what)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


class Scene:
    """Host lanes: lane_off int32 [L+1], length float32 [N]."""

    def __init__(self, lane_off, length):
        self.lane_off = np.ascontiguousarray(lane_off, dtype=np.int32)
        self.length = _f32(length)

    def c(self):
        return idm_cpu_scene_t(len(self.lane_off) - 1, len(self.length), _ptr(self.lane_off), _ptr(self.length))


def _params(theta):
    return idm_params_t(*[theta[q].ctypes.data for q in range(6)])


def max_threads():
    return load().idm_cpu_max_threads()


def idm_cpu_forward(theta, p_init, v_init, scene, K, dt, a_min=-10.0, threads=0, want_speed=False):
    """(K+1, N) positions (and speeds)."""
    theta, p_init, v_init = _f32(theta), _f32(p_init), _f32(v_init)
    N = len(scene.length)
    traj = np.empty((K + 1, N), np.float32)
    vtraj = np.empty((K + 1, N), np.float32) if want_speed else None
    _check(load().idm_cpu_forward(threads, ctypes.byref(scene.c()), ctypes.byref(_params(theta)), _ptr(p_init),
                                  _ptr(v_init), ctypes.byref(idm_sim_t(K, dt, a_min)), _ptr(traj), _ptr(vtraj)),
           "idm_cpu_forward")
    return (traj, vtraj) if want_speed else traj


def idm_cpu_loss_grad(theta, p_init, v_init, scene, K, dt, targets, obs_stride=1, a_min=-10.0, threads=0):
    """(loss, g_theta (6, N), g_p_init, g_v_init)."""
    theta, p_init, v_init = _f32(theta), _f32(p_init), _f32(v_init)
    targets = _f32(targets) if targets is not None else None
    N = len(scene.length)
    g = np.zeros((6, N), np.float32)
    gp, gv = np.zeros(N, np.float32), np.zeros(N, np.float32)
    loss = ctypes.c_double(0.0)
    _check(load().idm_cpu_loss_grad(threads, ctypes.byref(scene.c()), ctypes.byref(_params(theta)), _ptr(p_init),
                                    _ptr(v_init), ctypes.byref(idm_sim_t(K, dt, a_min)), _ptr(targets), obs_stride,
                                    ctypes.byref(loss), ctypes.byref(_params(g)), _ptr(gp), _ptr(gv)),
           "idm_cpu_loss_grad")
    return loss.value, g, gp, gv


def idm_cpu_fit(theta, p_init, v_init, scene, K, dt, targets, obs_stride, n_iter, lr0=0.1, lr1=0.01,
                box_lo=(20.0, 0.1, 1.0, 0.5, 0.1), box_hi=(60.0, 5.0, 10.0, 10.0, 5.0), a_min=-10.0, threads=0):
    """Adam fit in place on theta (float32 (6, N) C-contiguous); returns the loss history."""
    assert theta.dtype == np.float32 and theta.flags.c_contiguous
    p_init, v_init, targets = _f32(p_init), _f32(v_init), _f32(targets)
    hist = np.zeros(max(n_iter, 1))
    lo = (ctypes.c_float * 5)(*box_lo)
    hi = (ctypes.c_float * 5)(*box_hi)
    _check(load().idm_cpu_fit(threads, ctypes.byref(scene.c()), ctypes.byref(_params(theta)), _ptr(p_init),
                              _ptr(v_init), ctypes.byref(idm_sim_t(K, dt, a_min)), _ptr(targets), obs_stride, n_iter,
                              lr0, lr1, lo, hi, _ptr(hist)), "idm_cpu_fit")
    return hist[:n_iter]
