"""ctypes binding of libcollage (include/collage.h): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module converts numpy / torch arguments
into the C structs and pointers of the ABI, checks the returned status and raises with the
library's message.  There is no fallback: if libcollage.so cannot be loaded the import of the
binding fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcollage.so")
# COLLAGE_CHECKED=1 selects the bounds-checked build of the same sources (see build.py)
LIB_CHECKED_PATH = os.path.join(_HERE, "_build", "libcollage_checked.so")

COLLAGE_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "OVERFLOW", -5: "TIMEOUT", -6: "STATE"}
N_STAGES = 9
STAGES = ["transform", "bin", "raster_fwd", "composite", "dilate", "raster_bwd", "reduce", "loss",
          "adam"]

_ip = C.POINTER(C.c_int)
_fp = C.POINTER(C.c_float)
_up = C.POINTER(C.c_ubyte)


class collage_problem(C.Structure):
    _fields_ = [("n_elems", C.c_int), ("kind", _ip), ("pt_off", _ip), ("pts", _fp),
                ("stroke_hw", _fp), ("params0", _fp), ("trainable", _up), ("n_rings", C.c_int),
                ("ring_off", _ip), ("ring_pts", _fp), ("grid", C.c_int)]


class collage_options(C.Structure):
    _fields_ = [("alpha", C.c_float), ("beta", C.c_float), ("gamma", C.c_float),
                ("delta_down", C.c_float), ("tau", C.c_float), ("w_in", C.c_float),
                ("w_out", C.c_float), ("n_dilations", C.c_int), ("dil_weight", C.c_float * 8),
                ("pad_px", C.c_float), ("rho_px", C.c_float), ("segs_per_cubic", C.c_int),
                ("n_levels", C.c_int), ("level_res", C.c_int * 8), ("level_iters", C.c_int * 8),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("s_min", C.c_float), ("s_max", C.c_float), ("deterministic", C.c_int),
                ("tile", C.c_int), ("persistent", C.c_int), ("use_graphs", C.c_int),
                ("overlap_launches", C.c_int), ("force_kind", C.c_int), ("force_x", C.c_float),
                ("force_y", C.c_float), ("fit_controls", C.c_int)]


class collage_info(C.Structure):
    _fields_ = [("n_probs", C.c_int), ("n_elems", C.c_int), ("level", C.c_int),
                ("n_levels", C.c_int), ("tile", C.c_int), ("total_pixels", C.c_longlong),
                ("pair_capacity", C.c_int), ("last_pairs", C.c_int), ("kernels_per_iter", C.c_int),
                ("path_row_fallback", C.c_longlong), ("path_long_near", C.c_longlong),
                ("path_wide_tile", C.c_longlong), ("path_ring_chunk", C.c_longlong)]


class collage_tuning(C.Structure):
    _fields_ = [("tile", C.c_int), ("emit_threads", C.c_int), ("chunk_px", C.c_int), ("fwd_grid", C.c_float),
                ("bwd_grid", C.c_float), ("comp_grid", C.c_float), ("default_ms", C.c_float),
                ("best_ms", C.c_float), ("trials", C.c_int), ("from_cache", C.c_int)]


# name -> (restype, argtypes), the C ABI of include/collage.h
_vp = C.c_void_p
SIGNATURES = {
    "collage_default_options": (None, [C.POINTER(collage_options)]),
    "collage_create": (C.c_int, [C.POINTER(collage_problem), C.c_int, C.POINTER(collage_options),
                                 C.POINTER(_vp)]),
    "collage_set_level": (C.c_int, [_vp, C.c_int]),
    "collage_render": (C.c_int, [_vp, _vp, _vp, _vp]),
    "collage_loss_backward": (C.c_int, [_vp, _vp, _vp, _vp]),
    "collage_fp32_peak": (C.c_int, [_vp, C.c_void_p]),
    "collage_metrics": (C.c_int, [_vp, _vp, C.c_void_p]),
    "collage_step": (C.c_int, [_vp, _vp, C.c_int]),
    "collage_step_async": (C.c_int, [_vp, _vp, C.c_int]),
    "collage_run_schedule": (C.c_int, [_vp, _vp]),
    "collage_step_host": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp]),
    "collage_get_loss": (C.c_int, [_vp, _vp, _vp]),
    "collage_get_params": (C.c_int, [_vp, _vp, _vp]),
    "collage_set_params": (C.c_int, [_vp, _vp, _vp]),
    "collage_mat_init": (C.c_int, [_vp, _vp, _vp, _vp]),
    "collage_get_controls": (C.c_int, [_vp, _vp, _vp]),
    "collage_set_controls": (C.c_int, [_vp, _vp, _vp]),
    "collage_get_control_grad": (C.c_int, [_vp, _vp, _vp]),
    "collage_get_state": (C.c_int, [_vp, _vp, _vp, _ip, _ip]),
    "collage_set_state": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int]),
    "collage_get_bins": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _ip]),
    "collage_stage_times": (C.c_int, [_vp, _vp, C.c_int, _fp]),
    "collage_autotune": (C.c_int, [_vp, _vp, _fp]),
    "collage_get_tuning": (C.c_int, [_vp, C.POINTER(collage_tuning)]),
    "collage_set_tuning": (C.c_int, [_vp, _vp, C.POINTER(collage_tuning)]),
    "collage_uniform_term_noalloc": (C.c_int, [_vp, C.c_int, C.c_int, _fp, _vp, _vp, _vp, _vp]),
    "collage_get_info": (C.c_int, [_vp, C.POINTER(collage_info)]),
    "collage_sync": (C.c_int, [_vp, _vp]),
    "collage_last_error": (C.c_char_p, [_vp]),
    "collage_destroy": (None, [_vp]),
}

_lib = None


def load(path: str | None = None):
    """Load libcollage.so (built by paper_2406_04008_gb300.build), or its bounds-checked build when
    the environment sets COLLAGE_CHECKED=1, and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_CHECKED_PATH if os.environ.get("COLLAGE_CHECKED") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libcollage.so is not built ({path}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class CollageError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{ERRORS.get(status, status)}: {msg}")
        self.status = status


def check(status, handle=None):
    if status != COLLAGE_OK:
        msg = load().collage_last_error(handle)
        raise CollageError(status, msg.decode() if msg else "")


def default_options() -> collage_options:
    o = collage_options()
    load().collage_default_options(C.byref(o))
    return o


def make_options(**kw) -> collage_options:
    """Defaults of collage_default_options with keyword overrides; list fields take sequences."""
    o = default_options()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        if k in ("dil_weight", "level_res", "level_iters"):
            arr = getattr(o, k)
            for i in range(len(arr)):
                arr[i] = v[i] if i < len(v) else 0
        else:
            setattr(o, k, v)
    return o


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


class ProblemArrays:
    """Keeps the numpy arrays of one problem alive and exposes its collage_problem struct."""

    def __init__(self, prob: dict):
        self.kind = np.ascontiguousarray(prob["kind"], np.int32)
        self.pt_off = np.ascontiguousarray(prob["pt_off"], np.int32)
        self.pts = np.ascontiguousarray(prob["pts"], np.float32)
        self.hw = np.ascontiguousarray(prob["hw"], np.float32) if prob.get("hw") is not None else None
        self.params0 = np.ascontiguousarray(prob["params0"], np.float32)
        tr = prob.get("trainable")
        self.trainable = np.ascontiguousarray(tr, np.uint8) if tr is not None else None
        self.ring_off = np.ascontiguousarray(prob["ring_off"], np.int32)
        self.ring_pts = np.ascontiguousarray(prob["ring_pts"], np.float32)
        self.struct = collage_problem(
            n_elems=len(self.kind), kind=_ptr(self.kind, C.c_int), pt_off=_ptr(self.pt_off, C.c_int),
            pts=_ptr(self.pts, C.c_float), stroke_hw=_ptr(self.hw, C.c_float),
            params0=_ptr(self.params0, C.c_float), trainable=_ptr(self.trainable, C.c_ubyte),
            n_rings=len(self.ring_off) - 1, ring_off=_ptr(self.ring_off, C.c_int),
            ring_pts=_ptr(self.ring_pts, C.c_float), grid=int(prob.get("grid", 0)))
