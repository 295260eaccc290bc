"""ctypes loader for libqmcspl.so, the CUDA C-ABI library declared in include/qmcspl.h.

Argument marshalling only.  There is no fallback: if the library cannot be found or
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqmcspl.so")

OK = 0
ERR_ARG = 1
ERR_CUDA = 2
ERR_OOM = 3
ERR_UNSUPPORTED = 4
ERR_TIMEOUT = 5
ERR_NOT_HERMITIAN = 6
ERR_DEVICE = 7

BSPLINE_SMOOTH = 0
BSPLINE_INTERP = 1
LAGRANGE = 2
PPSPLINE = 3

F64 = 0
F32 = 1
BF16 = 2
DF64 = 3

MAX_BATCH = 48
NOALLOC_MAX_POS = 1 << 20
SLATER_MAX_BLOCK = 160
SLATER_MAX_COMPLEX_BLOCK = 112
SLATER_ARITH = {"f64": 0, "df64": 1}

ORDER_AUTO = 0
ORDER_INPUT = 1
ORDER_CELL = 2
ORDER_PENCIL = 3

METHODS = {"smooth": BSPLINE_SMOOTH, "interp": BSPLINE_INTERP, "lagrange": LAGRANGE, "pp": PPSPLINE}
STORAGE = {"f64": F64, "f32": F32, "bf16": BF16, "df64": DF64}


class QmcsplError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("qmcspl error %d: %s" % (code, msg))
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("storage", ctypes.c_int), ("separate_lap", ctypes.c_int),
                ("lanes", ctypes.c_int), ("separate_grad", ctypes.c_int), ("bloch", ctypes.c_int),
                ("kpoint", ctypes.c_double * 3)]


class Info(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 3), ("n_orb", ctypes.c_int), ("n_orb_padded", ctypes.c_int),
                ("method", ctypes.c_int), ("storage", ctypes.c_int), ("separate_lap", ctypes.c_int),
                ("n_tables", ctypes.c_int), ("entries_per_point", ctypes.c_int),
                ("rows_z", ctypes.c_int), ("lanes", ctypes.c_int), ("tiles", ctypes.c_int),
                ("table_bytes", ctypes.c_longlong), ("n_pw", ctypes.c_longlong),
                ("bloch", ctypes.c_int), ("kpoint", ctypes.c_double * 3), ("separate_grad", ctypes.c_int),
                ("degree", ctypes.c_int), ("nonuniform", ctypes.c_int), ("staged", ctypes.c_int),
                ("block_threads", ctypes.c_int)]


class HostOpts(ctypes.Structure):
    _fields_ = [("out_type", ctypes.c_int)]


OUT_TYPE = {"native": 0, "bf16": 1, "f16": 2}


class BatchOpts(ctypes.Structure):
    _fields_ = [("launch", ctypes.c_int), ("threads", ctypes.c_int)]


BATCH_LAUNCH = {"auto": 0, "single": 1, "split": 2}


class GridOpts(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("knots", ctypes.c_void_p * 3)]


_lock = threading.Lock()
_lib = None

VP = ctypes.c_void_p
LL = ctypes.c_longlong
I = ctypes.c_int

# (name, restype, argtypes) of every entry point of include/qmcspl.h
PROTOTYPES = [
    ("qmcspl_create", I, [ctypes.POINTER(VP), VP, VP, I, VP, I, VP, ctypes.POINTER(Opts), VP]),
    ("qmcspl_create_grid", I, [ctypes.POINTER(VP), VP, VP, I, VP, I, VP, ctypes.POINTER(Opts),
                               ctypes.POINTER(GridOpts), VP]),
    ("qmcspl_destroy", I, [VP]),
    ("qmcspl_info", I, [VP, ctypes.POINTER(Info)]),
    ("qmcspl_eval_vgl", I, [VP, VP, LL, VP, VP, VP, VP]),
    ("qmcspl_eval_vgl_host", I, [VP, VP, LL, VP, VP, VP, VP]),
    ("qmcspl_eval_vgl_host_ex", I, [VP, VP, LL, VP, VP, VP, ctypes.POINTER(HostOpts), VP]),
    ("qmcspl_eval_vgl_noalloc", I, [VP, VP, LL, VP, VP, VP, VP]),
    ("qmcspl_eval_vgl_backward", I, [VP, VP, LL, VP, VP, VP, VP, VP, VP, VP]),
    ("qmcspl_eval_batched", I, [I, VP, VP, VP, VP, VP, VP, VP]),
    ("qmcspl_eval_batched_ex", I, [I, VP, VP, VP, VP, VP, VP, ctypes.POINTER(BatchOpts), VP]),
    ("qmcspl_set_block", I, [VP, I]),
    ("qmcspl_get_table", I, [VP, I, VP, VP]),
    ("qmcspl_set_table", I, [VP, I, VP, I, VP]),
    ("qmcspl_set_order", I, [VP, I]),
    ("qmcspl_get_order", I, [VP, LL, ctypes.POINTER(I)]),
    ("qmcspl_profile", I, [VP, I]),
    ("qmcspl_profile_read", I, [VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_longlong)]),
    ("qmcspl_save", I, [VP, ctypes.c_char_p]),
    ("qmcspl_load", I, [ctypes.POINTER(VP), ctypes.c_char_p, VP]),
    ("qmcspl_slater_kinetic", I, [VP, VP, VP, I, I, LL, I, I, I, VP, VP, VP, VP, VP]),
    ("qmcspl_debug_fail_alloc", I, [LL]),
    ("qmcspl_debug_stall_pipeline", I, [I]),
    ("qmcspl_probe_cache", I, [I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), VP]),
    ("qmcspl_probe_fma", I, [I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), VP]),
    ("qmcspl_sync", I, [VP, VP]),
    ("qmcspl_last_error", ctypes.c_char_p, []),
    ("qmcspl_version", I, []),
]


def load(path: str = None):
    """Load the library (once) and attach the prototypes.  Raises if it is missing.
    QMCSPL_LIBRARY in the environment names another build of it (e.g. the bounds-checked
    libqmcspl_debug.so) to load instead."""
    global _lib
    path = path or os.environ.get("QMCSPL_LIBRARY") or LIB_PATH
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise QmcsplError(ERR_UNSUPPORTED,
                                  "libqmcspl.so not built (run __graft_entry__.build()): %s" % path)
            lib = ctypes.CDLL(path)
            for name, res, args in PROTOTYPES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int) -> None:
    if rc != OK:
        raise QmcsplError(rc, load().qmcspl_last_error().decode(errors="replace"))
