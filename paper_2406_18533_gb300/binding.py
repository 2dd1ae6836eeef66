"""ctypes binding of libgs (include/gs.h): the same entry points with the same
names, argument marshalling only.  Every step of the hot path runs in the
library's CUDA kernels; there is no Python or CPU fallback.  Loading raises
if ``libgs.so`` has not been built (``python -m paper_2406_18533_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")

c_float_p = ctypes.c_void_p


class gs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("W", ctypes.c_int32),
                ("H", ctypes.c_int32), ("near_z", ctypes.c_float), ("reserved", ctypes.c_int32)]


class gs_scene(ctypes.Structure):
    _fields_ = [("mo", ctypes.c_void_p), ("ls", ctypes.c_void_p), ("q", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gs_hparams(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("smem_batch", ctypes.c_int32), ("strict_nonfinite", ctypes.c_int32),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float), ("T_min", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("lr", ctypes.c_float * 6), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("scale_lr_sqrt_b", ctypes.c_int32),
                ("scale_beta_pow_b", ctypes.c_int32), ("lambda_dssim", ctypes.c_float),
                ("px_per_thread", ctypes.c_int32), ("sparse_adam", ctypes.c_int32),
                ("schedule", ctypes.c_int32)]


class gs_proj(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("conic_o", ctypes.c_void_p), ("rgb_d", ctypes.c_void_p),
                ("radius", ctypes.c_void_p), ("N", ctypes.c_int64), ("B", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class gs_proj_grad(ctypes.Structure):
    _fields_ = [("d_xy_o", ctypes.c_void_p), ("d_conic", ctypes.c_void_p), ("d_rgb", ctypes.c_void_p)]


class gs_bins(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
                ("count", ctypes.c_void_p), ("capacity", ctypes.c_uint64)]


class gs_densify_params(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("scale_threshold", ctypes.c_float),
                ("min_opacity", ctypes.c_float), ("split_div", ctypes.c_float)]


GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_NONFINITE, GS_ERR_OOM = range(7)
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA", 4: "GS_ERR_TIMEOUT",
                5: "GS_ERR_NONFINITE", 6: "GS_ERR_OOM"}
GS_MAX_VIEWS = 32

P = ctypes.POINTER
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64

# name -> argtypes (restype gs_status = int32 unless noted)
SIGNATURES = {
    "gs_create": [P(_vp), P(gs_hparams)],
    "gs_destroy": [_vp],
    "gs_default_hparams": [P(gs_hparams)],
    "gs_set_hparams": [_vp, P(gs_hparams)],
    "gs_last_error": [_vp],
    "gs_abi_version": [],
    "gs_reserve": [_vp, _i64, P(gs_camera), _i32, ctypes.c_uint64],
    "gs_workspace_size": [P(gs_hparams), _i64, P(gs_camera), _i32, ctypes.c_uint64, P(ctypes.c_size_t)],
    "gs_set_workspace": [_vp, _vp, ctypes.c_size_t, _vp],
    "gs_get_step": [_vp, P(_i64), _vp],
    "gs_set_step": [_vp, _i64, _vp],
    "gs_get_status": [_vp, _vp, P(_i32), P(ctypes.c_uint64)],
    "gs_get_counters": [_vp, _vp, P(ctypes.c_uint64)],
    "gs_count_work": [_vp, _i32],
    "gs_preprocess": [_vp, P(gs_scene), P(gs_camera), _i32, P(gs_proj), _vp],
    "gs_bin": [_vp, P(gs_proj), P(gs_camera), _i32, P(gs_bins), P(ctypes.c_uint64), _vp],
    "gs_render_fwd": [_vp, P(gs_proj), P(gs_bins), P(gs_camera), _i32, _vp, _vp, _vp, _vp],
    "gs_render_bwd": [_vp, P(gs_proj), P(gs_bins), P(gs_camera), _i32, _vp, _vp, _vp, P(gs_proj_grad), _vp],
    "gs_preprocess_bwd": [_vp, P(gs_scene), P(gs_camera), _i32, P(gs_proj), P(gs_proj_grad), P(gs_scene), _vp],
    "gs_preprocess_bwd_scaled": [_vp, P(gs_scene), P(gs_camera), _i32, P(gs_proj), P(gs_proj_grad), P(gs_scene),
                                 ctypes.c_float, _vp],
    "gs_loss": [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp],
    "gs_spatial_order": [_vp, P(gs_scene), _vp, _vp],
    "gs_division_points": [_vp, _vp, _i64, _i32, _vp, _vp],
    "gs_set_densify_stats": [_vp, _vp, _vp, _i64],
    "gs_densify": [_vp, P(gs_scene), P(gs_scene), P(gs_scene), _vp, _vp, _vp, P(gs_densify_params), P(gs_scene),
                   P(gs_scene), P(gs_scene), _i64, P(_i64), _vp],
    "gs_reset_opacity": [_vp, P(gs_scene), P(gs_scene), P(gs_scene), ctypes.c_float, _vp],
    "gs_permute": [_vp, P(gs_scene), _vp, P(gs_scene), _vp],
    "gs_adam_step_sparse": [_vp, P(gs_scene), P(gs_scene), P(gs_scene), P(gs_scene), _vp, _i64, _i32, _vp],
    "gs_adam_step": [_vp, P(gs_scene), P(gs_scene), P(gs_scene), P(gs_scene), _i64, _i32, _vp],
    "gs_train_step": [_vp, P(gs_scene), P(gs_scene), P(gs_scene), P(gs_scene), _i64, P(gs_camera), _i32, _vp, _vp,
                      _vp],
    "gs_render": [_vp, P(gs_scene), P(gs_camera), _i32, P(_vp), _vp],
    "gs_trace_enable": [_vp, _i32],
    "gs_trace_read": [_vp, P(ctypes.c_float), P(_i32)],
    "gs_kernel_launches": [],
    "gs_debug_set_lookback": [ctypes.c_uint32, _i32],
    "gs_debug_fail_alloc": [_i64],
    "gs_bin_noalloc": [P(gs_proj), P(gs_camera), _i32, _i32, P(gs_bins), P(ctypes.c_uint64), _vp],
}
NOALLOC_MAX_PAIRS = 1 << 18
NOALLOC_MAX_FRAGS = 1 << 20
GS_TRACE_STAGES = 11
TRACE_STAGES = ("preprocess", "order", "emit", "sort", "ranges", "blend_fwd", "loss", "zero_grad", "blend_bwd",
                "preprocess_bwd", "adam")

_lib = None
_lock = threading.Lock()


class GSError(RuntimeError):
    def __init__(self, name, status, text=""):
        super().__init__(f"{name} -> {STATUS_NAMES.get(status, status)}: {text}")
        self.status = status


def lib(path: str | None = None):
    """Load libgs.so (once).  Raises if it is missing: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libgs.so not built at {p}: run `python -m paper_2406_18533_gb300.build`")
            L = ctypes.CDLL(p)
            for name, argt in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = argt
                fn.restype = ctypes.c_int32
            L.gs_last_error.restype = ctypes.c_char_p
            L.gs_kernel_launches.restype = ctypes.c_uint64
            _lib = L
    return _lib


def call(name, *args, ctx=None):
    """Call an entry point; raise GSError on a non-OK status."""
    st = getattr(lib(), name)(*args)
    if st != GS_OK:
        text = lib().gs_last_error(ctx).decode() if ctx else ""
        raise GSError(name, st, text)
    return st


def camera_struct(cam) -> gs_camera:
    c = gs_camera()
    R = [float(x) for x in list(cam.R.reshape(9))]
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = float(cam.t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.W, c.H = int(cam.W), int(cam.H)
    c.near_z = float(cam.near)
    return c


def camera_array(cams):
    arr = (gs_camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


def default_hparams(**kw) -> gs_hparams:
    hp = gs_hparams()
    lib().gs_default_hparams(ctypes.byref(hp))
    for k, v in kw.items():
        if k in ("bg", "lr"):
            arr = getattr(hp, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(hp, k, v)
    return hp
