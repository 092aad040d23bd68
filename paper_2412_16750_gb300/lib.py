"""ctypes binding of libidm (include/idm.h): same names, argument marshalling only.

Every compute step runs inside libidm's CUDA kernels; this module only turns
Python values into C structs and raw pointers.  It raises ``RuntimeError``
when the library has not been built -- there is no CPU fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libidm.so")

IDM_OK = 0
IDM_ERR_ARG = 1
IDM_ERR_WORKSPACE = 2
IDM_ERR_CUDA = 3
IDM_ERR_NONFINITE = 4
IDM_ERR_TIMEOUT = 5
IDM_ERR_LANE = 6
IDM_ERR_OBS = 7
IDM_ERR_LANES = 8

IDM_STATUS_LANE_TOO_LONG = 1
IDM_STATUS_BAD_LANE_OFF = 2
IDM_STATUS_NONFINITE = 4
IDM_STATUS_TIMEOUT = 8
IDM_STATUS_BAD_OBS = 16
IDM_STATUS_BAD_LANES = 32

IDM_FIT_AUTO = 0
IDM_FIT_GRAPH = 1
IDM_FIT_SINGLE_LAUNCH = 2

IDM_MLP_IN = 80
IDM_MLP_HIDDEN = 256
IDM_MLP_OUT = 5
IDM_MLP_PREFIX = 20
IDM_MLP_N_PARAMS = 153605

GAP_FLOOR = 0.1
KINK_BAND = 0.5

_vp = ctypes.c_void_p


class idm_scene_t(ctypes.Structure):
    _fields_ = [("n_lanes", ctypes.c_int32), ("n_vehicles", ctypes.c_int32), ("max_lane", ctypes.c_int32),
                ("lane_off", _vp), ("length", _vp)]


class idm_params_t(ctypes.Structure):
    _fields_ = [("v0", _vp), ("T", _vp), ("s0", _vp), ("a_max", _vp), ("b", _vp), ("delta", _vp)]


class idm_sim_t(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("dt", ctypes.c_float), ("a_min", ctypes.c_float)]


class idm_batch_t(ctypes.Structure):
    _fields_ = [("n_scen", ctypes.c_int32), ("scen_lane_off", _vp), ("K", _vp), ("dt", _vp), ("obs_stride", _vp),
                ("a_min", ctypes.c_float), ("n_lanes", ctypes.c_int32), ("n_vehicles", ctypes.c_int32),
                ("lane_off_host", _vp), ("lane_off", _vp), ("length", _vp)]


class idm_recon_t(ctypes.Structure):
    _fields_ = [("n_traj", ctypes.c_int32), ("k_max", ctypes.c_int32), ("ld", ctypes.c_int32),
                ("n_obs", ctypes.c_int64), ("obs_off", _vp), ("obs_t", _vp), ("obs_p", _vp), ("obs_k", _vp),
                ("K", _vp), ("p_init", _vp), ("v_init", _vp), ("dt", ctypes.c_float), ("a_min", ctypes.c_float)]


class idm_lanes_t(ctypes.Structure):
    _fields_ = [("n_lanes", ctypes.c_int32), ("n_points", ctypes.c_int32), ("pt_off", _vp), ("px", _vp),
                ("py", _vp), ("lane_len", _vp)]


# name -> (restype, argtypes)
_SIGS = {
    "idm_ctx_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_size_t]),
    "idm_ctx_destroy": (ctypes.c_int, [_vp]),
    "idm_last_error": (ctypes.c_char_p, [_vp]),
    "idm_status": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint32), _vp]),
    "idm_set_event_counting": (ctypes.c_int, [_vp, ctypes.c_int]),
    "idm_event_counts": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "idm_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "idm_max_lane_supported": (ctypes.c_int, []),
    "idm_workspace_bytes": (ctypes.c_size_t, [_vp, ctypes.POINTER(idm_scene_t), ctypes.POINTER(idm_sim_t)]),
    "idm_layout": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "idm_gather": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int, ctypes.POINTER(_vp),
                                  ctypes.POINTER(_vp), _vp]),
    "idm_forward": (ctypes.c_int, [_vp, ctypes.POINTER(idm_scene_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                   ctypes.POINTER(idm_sim_t), _vp, _vp, _vp]),
    "idm_backward": (ctypes.c_int, [_vp, ctypes.POINTER(idm_scene_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                    ctypes.POINTER(idm_sim_t), _vp, _vp, ctypes.POINTER(idm_params_t), _vp, _vp,
                                    _vp]),
    "idm_loss_grad": (ctypes.c_int, [_vp, ctypes.POINTER(idm_scene_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                     ctypes.POINTER(idm_sim_t), _vp, ctypes.c_int32, _vp,
                                     ctypes.POINTER(idm_params_t), _vp, _vp, _vp]),
    "idm_gather_rows": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp]),
    "idm_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "idm_set_fit_mode": (ctypes.c_int, [_vp, ctypes.c_int]),
    "idm_last_fit_form": (ctypes.c_int, [_vp]),
    "idm_phase_times": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int32)]),
    "idm_batch_sizes": (ctypes.c_int, [ctypes.POINTER(idm_batch_t), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "idm_batch_forward": (ctypes.c_int, [_vp, ctypes.POINTER(idm_batch_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                         _vp, _vp]),
    "idm_batch_loss_grad": (ctypes.c_int, [_vp, ctypes.POINTER(idm_batch_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                           _vp, _vp, _vp, ctypes.POINTER(idm_params_t), _vp, _vp, _vp]),
    "idm_batch_fit": (ctypes.c_int, [_vp, ctypes.POINTER(idm_batch_t), ctypes.POINTER(idm_params_t), _vp, _vp, _vp,
                                     ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_float), _vp, _vp, _vp]),
    "idm_loss_grad_noalloc": (ctypes.c_int, [ctypes.POINTER(idm_scene_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                             ctypes.POINTER(idm_sim_t), _vp, ctypes.c_int32, _vp,
                                             ctypes.POINTER(idm_params_t), _vp, _vp, _vp, _vp]),
    "idm_fit": (ctypes.c_int, [_vp, ctypes.POINTER(idm_scene_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                               ctypes.POINTER(idm_sim_t), _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                               ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                               _vp, _vp]),
    # learned initializer (include/idm_mlp.h)
    "idm_gemm_bf16": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]),
    "idm_mlp_gelu_eval": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _vp]),
    "idm_mlp_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32]),
    "idm_mlp_destroy": (ctypes.c_int, [_vp]),
    "idm_mlp_last_error": (ctypes.c_char_p, [_vp]),
    "idm_mlp_set_weights": (ctypes.c_int, [_vp, _vp, _vp]),
    "idm_mlp_get_weights": (ctypes.c_int, [_vp, _vp, _vp]),
    "idm_mlp_status": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_uint32)]),
    "idm_mlp_clear_status": (ctypes.c_int, [_vp, _vp]),
    "idm_mlp_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "idm_mlp_features": (ctypes.c_int, [ctypes.POINTER(idm_scene_t), _vp, _vp, ctypes.POINTER(idm_sim_t), _vp,
                                        ctypes.c_int32, _vp, ctypes.c_int32, _vp, ctypes.POINTER(idm_params_t), _vp,
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _vp]),
    "idm_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp]),
    "idm_mlp_predict_params": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.POINTER(idm_params_t),
                                              ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _vp]),
    "idm_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp]),
    "idm_mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_float, _vp, _vp]),
    "idm_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                     ctypes.c_float, _vp, _vp]),
    "idm_fit_eval": (ctypes.c_int, [_vp, ctypes.POINTER(idm_scene_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                    ctypes.POINTER(idm_sim_t), _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                    ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                    _vp, _vp, _vp, _vp]),
    # lane geometry of the prediction (include/idm_lanes.h)
    "idm_lane_prepare": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]),
    "idm_lane_project": (ctypes.c_int, [_vp, ctypes.POINTER(idm_lanes_t), ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                        _vp, _vp, _vp, _vp, _vp, _vp]),
    "idm_lane_unproject": (ctypes.c_int, [_vp, ctypes.POINTER(idm_lanes_t), ctypes.c_int32, ctypes.c_int32, _vp,
                                          _vp, _vp, _vp, _vp]),
    "idm_rollout_state": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                         _vp, _vp, _vp]),
    "idm_displacement": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_float, _vp,
                                        _vp, _vp, _vp]),
    # single-trajectory reconstruction mode (include/idm_recon.h)
    "idm_recon_prepare": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_float, _vp,
                                         _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int32), _vp]),
    "idm_recon_forward": (ctypes.c_int, [_vp, ctypes.POINTER(idm_recon_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                         _vp, _vp, _vp, _vp]),
    "idm_recon_loss_grad": (ctypes.c_int, [_vp, ctypes.POINTER(idm_recon_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                           _vp, ctypes.POINTER(idm_params_t), _vp, _vp, _vp, _vp, _vp]),
    "idm_recon_fit": (ctypes.c_int, [_vp, ctypes.POINTER(idm_recon_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                     ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_float), _vp, _vp]),
    "idm_recon_metrics": (ctypes.c_int, [_vp, ctypes.POINTER(idm_recon_t), ctypes.POINTER(idm_params_t), _vp, _vp,
                                         _vp, _vp]),
}

_lib = None


def exported_symbols():
    """Names the header declares (the binding's table)."""
    return sorted(_SIGS)


def load(path=None):
    """Load libidm.so; raises RuntimeError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libidm.so is not built (%s); run __graft_entry__.build() -- there is no CPU "
                           "fallback" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IdmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libidm error %d: %s" % (code, msg))
        self.code = code


def check(ctx, rc):
    if rc != IDM_OK:
        msg = load().idm_last_error(ctx)
        raise IdmError(rc, msg.decode() if msg else "")
    return rc


def ptr(t):
    """Raw device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream)


# ---- same-name thin wrappers ------------------------------------------------

def idm_ctx_create(workspace_cap_bytes=0):
    h = _vp()
    rc = load().idm_ctx_create(ctypes.byref(h), workspace_cap_bytes)
    if rc != IDM_OK:
        raise IdmError(rc, "idm_ctx_create failed")
    return h


def idm_ctx_destroy(ctx):
    return load().idm_ctx_destroy(ctx)


def idm_last_error(ctx):
    m = load().idm_last_error(ctx)
    return m.decode() if m else ""


def idm_status(ctx, stream=None):
    flags = ctypes.c_uint32(0)
    rc = load().idm_status(ctx, ctypes.byref(flags), stream_ptr(stream))
    return rc, flags.value


def idm_set_event_counting(ctx, on):
    return check(ctx, load().idm_set_event_counting(ctx, 1 if on else 0))


def idm_event_counts(ctx, stream=None):
    """(gap_floor_hits, kink_near) since the last read; clears them."""
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    check(ctx, load().idm_event_counts(ctx, stream_ptr(stream), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def idm_set_tuning(ctx, vpt=0, warps_per_segment=0, ckpt_interval=8, warps_per_block=8):
    return check(ctx, load().idm_set_tuning(ctx, vpt, warps_per_segment, ckpt_interval, warps_per_block))


def idm_max_lane_supported():
    return load().idm_max_lane_supported()


def idm_workspace_bytes(ctx, scene, sim):
    return load().idm_workspace_bytes(ctx, ctypes.byref(scene), ctypes.byref(sim))


def idm_layout(ctx, N, n_lanes, lane_id, pos, perm, lane_off, max_lane_out=None, stream=None):
    return check(ctx, load().idm_layout(ctx, N, n_lanes, ptr(lane_id), ptr(pos), ptr(perm), ptr(lane_off),
                                        ptr(max_lane_out), stream_ptr(stream)))


def idm_gather(ctx, N, perm, srcs, dsts, stream=None):
    n = len(srcs)
    s = (_vp * max(n, 1))(*[t.data_ptr() for t in srcs])
    d = (_vp * max(n, 1))(*[t.data_ptr() for t in dsts])
    return check(ctx, load().idm_gather(ctx, N, ptr(perm), n, s, d, stream_ptr(stream)))


def idm_gather_rows(ctx, N, n_rows, perm, src, dst, stream=None):
    return check(ctx, load().idm_gather_rows(ctx, N, n_rows, ptr(perm), ptr(src), ptr(dst), stream_ptr(stream)))


def idm_set_profiling(ctx, on):
    return check(ctx, load().idm_set_profiling(ctx, 1 if on else 0))


def idm_set_fit_mode(ctx, mode):
    return check(ctx, load().idm_set_fit_mode(ctx, int(mode)))


def idm_last_fit_form(ctx):
    return load().idm_last_fit_form(ctx)


def idm_phase_times(ctx, stream=None):
    f, b, n = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int32(0)
    check(ctx, load().idm_phase_times(ctx, stream_ptr(stream), ctypes.byref(f), ctypes.byref(b), ctypes.byref(n)))
    return f.value, b.value, n.value


def idm_forward(ctx, scene, params, p_init, v_init, sim, traj=None, vtraj=None, stream=None):
    return check(ctx, load().idm_forward(ctx, ctypes.byref(scene), ctypes.byref(params), ptr(p_init), ptr(v_init),
                                         ctypes.byref(sim), ptr(traj), ptr(vtraj), stream_ptr(stream)))


def idm_backward(ctx, scene, params, p_init, v_init, sim, gP, gV=None, grad=None, grad_p_init=None,
                 grad_v_init=None, stream=None):
    return check(ctx, load().idm_backward(ctx, ctypes.byref(scene), ctypes.byref(params), ptr(p_init),
                                          ptr(v_init), ctypes.byref(sim), ptr(gP), ptr(gV),
                                          ctypes.byref(grad) if grad is not None else None, ptr(grad_p_init),
                                          ptr(grad_v_init), stream_ptr(stream)))


def idm_loss_grad(ctx, scene, params, p_init, v_init, sim, targets, obs_stride, loss_out=None, grad=None,
                  grad_p_init=None, grad_v_init=None, stream=None):
    return check(ctx, load().idm_loss_grad(ctx, ctypes.byref(scene), ctypes.byref(params), ptr(p_init),
                                           ptr(v_init), ctypes.byref(sim), ptr(targets), obs_stride,
                                           ptr(loss_out), ctypes.byref(grad) if grad is not None else None,
                                           ptr(grad_p_init), ptr(grad_v_init), stream_ptr(stream)))


def idm_loss_grad_noalloc(scene, params, p_init, v_init, sim, targets, obs_stride, loss_out=None, grad=None,
                          grad_p_init=None, grad_v_init=None, status_out=None, stream=None):
    """Returns the raw status code (there is no context to hold a message)."""
    return load().idm_loss_grad_noalloc(ctypes.byref(scene), ctypes.byref(params), ptr(p_init), ptr(v_init),
                                        ctypes.byref(sim), ptr(targets), obs_stride, ptr(loss_out),
                                        ctypes.byref(grad) if grad is not None else None, ptr(grad_p_init),
                                        ptr(grad_v_init), ptr(status_out), stream_ptr(stream))


def idm_fit(ctx, scene, params, p_init, v_init, sim, targets, obs_stride, n_iter, lr0, lr1, box_lo, box_hi,
            loss_hist=None, stream=None):
    lo = (ctypes.c_float * 5)(*box_lo)
    hi = (ctypes.c_float * 5)(*box_hi)
    return check(ctx, load().idm_fit(ctx, ctypes.byref(scene), ctypes.byref(params), ptr(p_init), ptr(v_init),
                                     ctypes.byref(sim), ptr(targets), obs_stride, n_iter, lr0, lr1, lo, hi,
                                     ptr(loss_hist), stream_ptr(stream)))


def idm_fit_eval(ctx, scene, params, p_init, v_init, sim, targets, obs_stride, n_iter, lr0, lr1, box_lo, box_hi,
                 loss_hist=None, eval_targets=None, eval_hist=None, stream=None):
    lo = (ctypes.c_float * 5)(*box_lo)
    hi = (ctypes.c_float * 5)(*box_hi)
    return check(ctx, load().idm_fit_eval(ctx, ctypes.byref(scene), ctypes.byref(params), ptr(p_init), ptr(v_init),
                                          ctypes.byref(sim), ptr(targets), obs_stride, n_iter, lr0, lr1, lo, hi,
                                          ptr(loss_hist), ptr(eval_targets), ptr(eval_hist), stream_ptr(stream)))


def idm_batch_sizes(batch, ckpt_interval=8):
    t, y, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    rc = load().idm_batch_sizes(ctypes.byref(batch), ckpt_interval, ctypes.byref(t), ctypes.byref(y), ctypes.byref(c))
    if rc != IDM_OK:
        raise IdmError(rc, "idm_batch_sizes: bad batch description")
    return t.value, y.value, c.value


def idm_batch_forward(ctx, batch, params, p_init, v_init, traj, stream=None):
    return check(ctx, load().idm_batch_forward(ctx, ctypes.byref(batch), ctypes.byref(params), ptr(p_init),
                                               ptr(v_init), ptr(traj), stream_ptr(stream)))


def idm_batch_loss_grad(ctx, batch, params, p_init, v_init, targets, scen_loss=None, loss_total=None, grad=None,
                        grad_p_init=None, grad_v_init=None, stream=None):
    return check(ctx, load().idm_batch_loss_grad(ctx, ctypes.byref(batch), ctypes.byref(params), ptr(p_init),
                                                 ptr(v_init), ptr(targets), ptr(scen_loss), ptr(loss_total),
                                                 ctypes.byref(grad) if grad is not None else None,
                                                 ptr(grad_p_init), ptr(grad_v_init), stream_ptr(stream)))


def idm_batch_fit(ctx, batch, params, p_init, v_init, targets, n_iter, lr0, lr1, box_lo, box_hi, loss_hist=None,
                  scen_loss=None, stream=None):
    lo = (ctypes.c_float * 5)(*box_lo)
    hi = (ctypes.c_float * 5)(*box_hi)
    return check(ctx, load().idm_batch_fit(ctx, ctypes.byref(batch), ctypes.byref(params), ptr(p_init), ptr(v_init),
                                           ptr(targets), n_iter, lr0, lr1, lo, hi, ptr(loss_hist), ptr(scen_loss),
                                           stream_ptr(stream)))


# ---- struct builders ---------------------------------------------------------

def idm_lane_prepare(ctx, n_lanes, n_points, pt_off, px, py, lane_len_out, stream=None):
    return check(ctx, load().idm_lane_prepare(ctx, n_lanes, n_points, ptr(pt_off), ptr(px), ptr(py),
                                              ptr(lane_len_out), stream_ptr(stream)))


def idm_lane_project(ctx, lanes, n_rows, n_cols, qx, qy, lane_lo, lane_hi=None, lane_out=None, s_out=None,
                     d_out=None, stream=None):
    return check(ctx, load().idm_lane_project(ctx, ctypes.byref(lanes), n_rows, n_cols, ptr(qx), ptr(qy), ptr(lane_lo),
                                              ptr(lane_hi), ptr(lane_out), ptr(s_out), ptr(d_out),
                                              stream_ptr(stream)))


def idm_lane_unproject(ctx, lanes, n_rows, n_cols, s, lane_of_col, x_out, y_out, stream=None):
    return check(ctx, load().idm_lane_unproject(ctx, ctypes.byref(lanes), n_rows, n_cols, ptr(s), ptr(lane_of_col),
                                                ptr(x_out), ptr(y_out), stream_ptr(stream)))


def idm_rollout_state(ctx, N, s_rows, row_a, row_b, dt, p_out, v_out, stream=None):
    return check(ctx, load().idm_rollout_state(ctx, N, ptr(s_rows), row_a, row_b, dt, ptr(p_out), ptr(v_out),
                                               stream_ptr(stream)))


def idm_displacement(ctx, F, N, px, py, tx, ty, miss_m, ade=None, fde=None, sums=None, stream=None):
    return check(ctx, load().idm_displacement(ctx, F, N, ptr(px), ptr(py), ptr(tx), ptr(ty), miss_m, ptr(ade),
                                              ptr(fde), ptr(sums), stream_ptr(stream)))


def idm_recon_prepare(ctx, N, n_obs, obs_off, obs_t, obs_p, dt, obs_k, K, p_init, v_init, want_k_max=True,
                      stream=None):
    """Returns max K (the call then waits for the stream) or None."""
    km = ctypes.c_int32(0)
    check(ctx, load().idm_recon_prepare(ctx, N, n_obs, ptr(obs_off), ptr(obs_t), ptr(obs_p), dt, ptr(obs_k), ptr(K),
                                        ptr(p_init), ptr(v_init), ctypes.byref(km) if want_k_max else None,
                                        stream_ptr(stream)))
    return km.value if want_k_max else None


def idm_recon_forward(ctx, rec, params, dp, dv, P=None, V=None, A=None, stream=None):
    return check(ctx, load().idm_recon_forward(ctx, ctypes.byref(rec), ctypes.byref(params), ptr(dp), ptr(dv),
                                               ptr(P), ptr(V), ptr(A), stream_ptr(stream)))


def idm_recon_loss_grad(ctx, rec, params, dp, dv, loss_out=None, grad=None, g_dp=None, g_dv=None, g_p_init=None,
                        g_v_init=None, stream=None):
    return check(ctx, load().idm_recon_loss_grad(ctx, ctypes.byref(rec), ctypes.byref(params), ptr(dp), ptr(dv),
                                                 ptr(loss_out), ctypes.byref(grad) if grad is not None else None,
                                                 ptr(g_dp), ptr(g_dv), ptr(g_p_init), ptr(g_v_init),
                                                 stream_ptr(stream)))


def idm_recon_fit(ctx, rec, params, dp, dv, n_iter, lr0, lr1, box_lo, box_hi, loss_hist=None, stream=None):
    lo = (ctypes.c_float * 5)(*box_lo)
    hi = (ctypes.c_float * 5)(*box_hi)
    return check(ctx, load().idm_recon_fit(ctx, ctypes.byref(rec), ctypes.byref(params), ptr(dp), ptr(dv), n_iter,
                                           lr0, lr1, lo, hi, ptr(loss_hist), stream_ptr(stream)))


def idm_recon_metrics(ctx, rec, params, dp, dv, out, stream=None):
    return check(ctx, load().idm_recon_metrics(ctx, ctypes.byref(rec), ctypes.byref(params), ptr(dp), ptr(dv),
                                               ptr(out), stream_ptr(stream)))


def make_scene(lane_off, length, max_lane):
    """lane_off (int32 CUDA tensor [L+1]), length (float32 CUDA tensor [N])."""
    return idm_scene_t(lane_off.numel() - 1, length.numel(), int(max_lane), lane_off.data_ptr(),
                       length.data_ptr())


def make_params(theta):
    """theta: float32 CUDA tensor (6, N), rows v0, T, s0, a_max, b, delta (contiguous rows).
    The row pointers come from the base pointer and the row stride (no row
    views are created: six views cost tens of microseconds per call)."""
    if theta.dim() == 2 and theta.stride(1) == 1:
        base, step = theta.data_ptr(), theta.stride(0) * theta.element_size()
        return idm_params_t(*[base + q * step for q in range(6)])
    return idm_params_t(*[theta[q].data_ptr() for q in range(6)])


def make_sim(K, dt, a_min=-10.0):
    return idm_sim_t(int(K), float(dt), float(a_min))


# ---- learned initializer (include/idm_mlp.h) --------------------------------

def _box(v):
    return (ctypes.c_float * 5)(*v) if v is not None else None


def mcheck(mlp, rc):
    if rc != IDM_OK:
        msg = load().idm_mlp_last_error(mlp)
        raise IdmError(rc, msg.decode() if msg else "")
    return rc


def idm_gemm_bf16(A, B, M, N, K, C, status, stream=None):
    """Raw status code (no object to hold a message)."""
    return load().idm_gemm_bf16(ptr(A), ptr(B), M, N, K, ptr(C), ptr(status), stream_ptr(stream))


def idm_mlp_gelu_eval(z, gelu_out=None, gelu_grad_out=None, stream=None):
    """Raw status code."""
    return load().idm_mlp_gelu_eval(ptr(z), ptr(gelu_out), ptr(gelu_grad_out), z.numel(), stream_ptr(stream))


def idm_mlp_create(max_batch):
    h = _vp()
    rc = load().idm_mlp_create(ctypes.byref(h), max_batch)
    if rc != IDM_OK:
        raise IdmError(rc, "idm_mlp_create failed")
    return h


def idm_mlp_destroy(mlp):
    return load().idm_mlp_destroy(mlp)


def idm_mlp_last_error(mlp):
    m = load().idm_mlp_last_error(mlp)
    return m.decode() if m else ""


def idm_mlp_set_weights(mlp, weights, stream=None):
    return mcheck(mlp, load().idm_mlp_set_weights(mlp, ptr(weights), stream_ptr(stream)))


def idm_mlp_get_weights(mlp, weights, stream=None):
    return mcheck(mlp, load().idm_mlp_get_weights(mlp, ptr(weights), stream_ptr(stream)))


def idm_mlp_status(mlp, stream=None):
    bits = ctypes.c_uint32(0)
    rc = load().idm_mlp_status(mlp, stream_ptr(stream), ctypes.byref(bits))
    return rc, bits.value


def idm_mlp_clear_status(mlp, stream=None):
    return mcheck(mlp, load().idm_mlp_clear_status(mlp, stream_ptr(stream)))


def idm_mlp_set_wait_limit(mlp, polls):
    return mcheck(mlp, load().idm_mlp_set_wait_limit(mlp, int(polls)))


def idm_mlp_features(scene, p_init, v_init, sim, targets, obs_stride, perm, n_rows, X, label_params=None,
                     labels=None, box_lo=None, box_hi=None, stream=None):
    rc = load().idm_mlp_features(ctypes.byref(scene), ptr(p_init), ptr(v_init), ctypes.byref(sim), ptr(targets),
                                 obs_stride, ptr(perm), n_rows, ptr(X),
                                 ctypes.byref(label_params) if label_params is not None else None, ptr(labels),
                                 _box(box_lo), _box(box_hi), stream_ptr(stream))
    if rc != IDM_OK:
        raise IdmError(rc, "idm_mlp_features: bad arguments")
    return rc


def idm_mlp_forward(mlp, X, B, out, stream=None):
    return mcheck(mlp, load().idm_mlp_forward(mlp, ptr(X), B, ptr(out), stream_ptr(stream)))


def idm_mlp_predict_params(mlp, X, B, params, box_lo, box_hi, stream=None):
    return mcheck(mlp, load().idm_mlp_predict_params(mlp, ptr(X), B, ctypes.byref(params), _box(box_lo),
                                                     _box(box_hi), stream_ptr(stream)))


def idm_mlp_loss_grad(mlp, X, labels, B, loss_out, grad, stream=None):
    return mcheck(mlp, load().idm_mlp_loss_grad(mlp, ptr(X), ptr(labels), B, ptr(loss_out), ptr(grad),
                                                stream_ptr(stream)))


def idm_mlp_train_step(mlp, X, labels, B, lr, loss_out=None, stream=None):
    return mcheck(mlp, load().idm_mlp_train_step(mlp, ptr(X), ptr(labels), B, lr, ptr(loss_out),
                                                 stream_ptr(stream)))


def idm_mlp_train(mlp, X, labels, n_samples, batch, n_steps, lr0, lr1, loss_hist=None, stream=None):
    return mcheck(mlp, load().idm_mlp_train(mlp, ptr(X), ptr(labels), n_samples, batch, n_steps, lr0, lr1,
                                            ptr(loss_hist), stream_ptr(stream)))
