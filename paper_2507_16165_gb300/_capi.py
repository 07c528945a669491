"""ctypes mirror of include/bh.h (argument marshalling only).

Every computation happens in libbh.so; this module only lays out the C
structures and converts Python / torch arguments to pointers.  Loading fails
loudly when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbh.so")

BH_MAX_SPHERES = 8
BH_MAX_HOST_STRIPS = 16
BH_OK = 0
BH_E_INVALID, BH_E_NOMEM, BH_E_CUDA, BH_E_DEVICE = -1, -2, -3, -4
BH_E_NO_SURROGATE, BH_E_IO, BH_E_UNSUPPORTED = -5, -6, -7
BH_MODE_FP64, BH_MODE_FP32, BH_MODE_MIXED, BH_MODE_SURROGATE = 0, 1, 2, 3
BH_MODE_PAPER_EPS, BH_MODE_PAPER_EPS_FP32 = 4, 5
BH_IC_STATIC, BH_IC_EUCLIDEAN = 0, 1
BH_FLAG_ESC, BH_FLAG_CAPT, BH_FLAG_DISK, BH_FLAG_SPHERE = 1, 2, 4, 8
BH_FLAG_BAND, BH_FLAG_FP64, BH_FLAG_SURR, BH_FLAG_STEP_LIMIT = 16, 32, 64, 128
BH_STATUS_ABORTED, BH_STATUS_WATCHDOG = 1, 2

MODES = {"fp64": BH_MODE_FP64, "fp32": BH_MODE_FP32, "mixed": BH_MODE_MIXED,
         "surrogate": BH_MODE_SURROGATE, "paper": BH_MODE_PAPER_EPS,
         "paper_fp32": BH_MODE_PAPER_EPS_FP32}


class bh_sphere(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("albedo", ctypes.c_double * 3)]


class bh_scene_desc(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("disk_enabled", ctypes.c_int),
                ("disk_r_in", ctypes.c_double), ("disk_r_out", ctypes.c_double),
                ("n_spheres", ctypes.c_int), ("spheres", bh_sphere * BH_MAX_SPHERES),
                ("sky_seed", ctypes.c_uint64), ("ic", ctypes.c_int)]


class bh_camera(ctypes.Structure):
    _fields_ = [("r_obs", ctypes.c_double), ("incl_deg", ctypes.c_double),
                ("azim_deg", ctypes.c_double), ("fov_deg", ctypes.c_double),
                ("pos", ctypes.c_double * 3), ("fwd", ctypes.c_double * 3),
                ("right", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("tan_half", ctypes.c_double)]


class bh_render_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("band", ctypes.c_double), ("band_rtol", ctypes.c_double),
                ("phi_max", ctypes.c_double),
                ("max_steps", ctypes.c_int), ("h_max", ctypes.c_double),
                ("stream", ctypes.c_void_p),
                ("block_size", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("budget", ctypes.c_int),
                ("periastron_reset", ctypes.c_int), ("abort_after", ctypes.c_uint32),
                ("h_max_far", ctypes.c_double), ("paper_eps", ctypes.c_double),
                ("spp", ctypes.c_int), ("doppler", ctypes.c_int),
                ("rtol_far", ctypes.c_double), ("host_strips", ctypes.c_int),
                ("rtol_near", ctypes.c_double), ("queue_chunk", ctypes.c_int)]


class bh_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "rays", "steps", "rejected", "n_esc", "n_capt", "n_disk", "n_sphere", "n_step_limit",
        "n_band", "n_long", "n_surrogate", "n_fallback", "queue_grabs", "periastron",
        "events", "steps_fp64")] + [("status", ctypes.c_uint32),
                                    ("kernel_ms", ctypes.c_float * 4),
                                    ("mlp_rays", ctypes.c_uint64)]


class bh_train_opts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("val_fraction", ctypes.c_double),
                ("err_threshold", ctypes.c_double), ("r_err_threshold", ctypes.c_double),
                ("stream", ctypes.c_void_p)]


class bh_train_report(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int), ("n_valid", ctypes.c_int), ("n_train", ctypes.c_int),
                ("n_val", ctypes.c_int), ("steps", ctypes.c_int), ("final_loss", ctypes.c_float),
                ("val_rmse", ctypes.c_float * 3), ("served_fraction", ctypes.c_float),
                ("label_ms", ctypes.c_float), ("train_ms", ctypes.c_float),
                ("calib_ms", ctypes.c_float)]


class bh_calib_opts(ctypes.Structure):
    _fields_ = [("nb_lb", ctypes.c_int), ("nb_r", ctypes.c_int),
                ("err_threshold", ctypes.c_double), ("r_err_threshold", ctypes.c_double),
                ("stream", ctypes.c_void_p)]


BH_MLP_NPARAM = 10448


class bh_tune_result(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("budget", ctypes.c_int),
                ("ms_best", ctypes.c_float), ("ms_default", ctypes.c_float),
                ("trials", ctypes.c_int), ("queue_chunk", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("bh_version", _I, []),
    ("bh_last_error", ctypes.c_char_p, []),
    ("bh_scene_create", _I, [ctypes.POINTER(bh_scene_desc), ctypes.POINTER(_P)]),
    ("bh_scene_destroy", None, [_P]),
    ("bh_scene_sky_texture", _I, [_P, _P, _I, _I]),
    ("bh_camera_set", _I, [ctypes.POINTER(bh_camera), ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, ctypes.c_double]),
    ("bh_render", _I, [_P, ctypes.POINTER(bh_camera), _I, _P, _P, _P, _P, _P,
                       ctypes.POINTER(bh_render_opts)]),
    ("bh_render_host", _I, [_P, ctypes.POINTER(bh_camera), _I, _P, _P, _P, _P, _P,
                            ctypes.POINTER(bh_render_opts)]),
    ("bh_scene_sync", _I, [_P]),
    ("bh_render_stats", _I, [_P, ctypes.POINTER(bh_stats)]),
    ("bh_graph_create", _I, [_P, ctypes.POINTER(bh_camera), _I, _P, _P, _P, _P, _P,
                             ctypes.POINTER(bh_render_opts), ctypes.POINTER(_P)]),
    ("bh_graph_launch", _I, [_P, _P]),
    ("bh_graph_destroy", None, [_P]),
    ("bh_autotune", _I, [_P, ctypes.POINTER(bh_camera), _I, _P, _P, _P, _P, _P,
                         ctypes.POINTER(bh_render_opts), ctypes.POINTER(bh_tune_result)]),
    ("bh_autotune_reset", _I, []),
    ("bh_surrogate_labels", _I, [ctypes.c_double, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("bh_surrogate_train", _I, [_P, _I, _P, _P, _P, ctypes.POINTER(bh_train_opts),
                                ctypes.POINTER(bh_train_report)]),
    ("bh_surrogate_calibrate", _I, [_P, _I, _P, _P, _P, ctypes.POINTER(bh_calib_opts), _P, _P,
                                    _P, _P]),
    ("bh_surrogate_get", _I, [_P, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("bh_surrogate_save", _I, [_P, ctypes.c_char_p]),
    ("bh_surrogate_load", _I, [_P, ctypes.c_char_p]),
    ("bh_mlp_grad", _I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    ("bh_mlp_infer", _I, [_P, _I, _P, _P, _P]),
    ("bh_selftest_wait_timeout", _I, [_I, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
    ("bh_render_noalloc", _I, [ctypes.POINTER(bh_scene_desc), ctypes.POINTER(bh_camera), _I,
                               _P, _P, _P, _P, _P, ctypes.POINTER(bh_render_opts)]),
]
BH_NOALLOC_MAX_CAMERAS = 64


def lib(path: str = LIB_PATH) -> ctypes.CDLL:
    """The loaded renderer library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA extension first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


class BHError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().bh_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def check(rc: int, where: str) -> None:
    if rc != BH_OK:
        raise BHError(rc, where)
