"""ctypes binding of libburgers (include/burgers.h): argument marshalling only.

Every function of the C ABI is exposed under its own name. There is no
fallback: if libburgers.so is missing or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libburgers.so")

BURGERS_OK = 0
BURGERS_EINVAL = 1
BURGERS_ENOMEM = 2
BURGERS_ECUDA = 3
BURGERS_EAGAIN = 4
BURGERS_ETIMEOUT = 5
BURGERS_ECANCELED = 6
BURGERS_ENOTFOUND = 7
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EAGAIN", 5: "ETIMEOUT",
                6: "ECANCELED", 7: "ENOTFOUND"}

BURGERS_F32 = 0
BURGERS_F64 = 1
BURGERS_PERIODIC = 0
BURGERS_DIRICHLET = 1
BURGERS_EXPLICIT = 0
BURGERS_BTCS = 1
BURGERS_RK4 = 2
BURGERS_CN = 3
BURGERS_PICARD = 4
BURGERS_NEWTON = 5

BURGERS_OPT_GRAPHS = 0
BURGERS_OPT_PLAIN = 1
BURGERS_OPT_STREAM_K = 2
BURGERS_OPT_RESIDENT_MAX = 3
BURGERS_OPT_AUTOTUNE = 4
BURGERS_OPT_LAUNCH_COUNT = 5
BURGERS_OPT_CLUSTER = 6
BURGERS_INFO_SM_COUNT = 100
BURGERS_INFO_CLUSTER_CTAS_MAX = 101

# numpy mirror of burgers_instance (48 bytes, natural alignment)
INSTANCE_DTYPE = np.dtype([("offset", "<i8"), ("n", "<i4"), ("bc", "<i4"), ("dx", "<f8"),
                           ("nu", "<f8"), ("dt", "<f8"), ("nsteps", "<i8")], align=True)


class burgers_instance(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_int64), ("n", ctypes.c_int32), ("bc", ctypes.c_int32),
                ("dx", ctypes.c_double), ("nu", ctypes.c_double), ("dt", ctypes.c_double),
                ("nsteps", ctypes.c_int64)]


class burgers_batch(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("count", ctypes.c_int64), ("inst", ctypes.c_void_p)]


assert ctypes.sizeof(burgers_instance) == INSTANCE_DTYPE.itemsize == 48

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_ST = ctypes.c_int

# name -> (restype, argtypes); every entry point declared in include/burgers.h
SIGNATURES = {
    "burgers_ctx_create": (_ST, [ctypes.c_int, ctypes.POINTER(_P)]),
    "burgers_ctx_destroy": (None, [_P]),
    "burgers_last_error": (ctypes.c_char_p, []),
    "burgers_ctx_set": (_ST, [_P, _I32, _I64]),
    "burgers_ctx_get": (_ST, [_P, _I32, ctypes.POINTER(ctypes.c_int64)]),
    "burgers_launch_count": (_I64, [_P]),
    "burgers_device_error": (_ST, [_P, _P, _I32]),
    "burgers_cfl_dt": (_ST, [_P, _P, _P, _D, _P, _P]),
    "burgers_cfl_dt_device": (_ST, [_P, _P, _P, _D, _P, _P]),
    "burgers_advance_dt_device": (_ST, [_P, _I32, _P, _P, _P, _D, _I32, _P]),
    "burgers_explicit_advance": (_ST, [_P, _P, _P, _P]),
    "burgers_btcs_advance": (_ST, [_P, _P, _P, _P]),
    "burgers_rk4_advance": (_ST, [_P, _P, _P, _P]),
    "burgers_cn_advance": (_ST, [_P, _P, _P, _P]),
    "burgers_picard_advance": (_ST, [_P, _P, _P, ctypes.c_int32, _P]),
    "burgers_newton_advance": (_ST, [_P, _P, _P, ctypes.c_int32, _P]),
    "burgers_solve_host": (_ST, [_P, _I32, _P, _P, _P]),
    "burgers_rel_l2": (_ST, [_P, _P, _P, _P, _I32, _P, _P, _P]),
    "burgers_fma_peak": (_ST, [_P, _I32, _P]),
    "burgers_adjoint": (_ST, [_P, _I32, _P, _P, _P, _P, _P, _I64, _P]),
    "burgers_autotune": (_ST, [_P, _I32, _P, _P, _I64, _P, _P]),
    "burgers_explicit_advance_noalloc": (_ST, [_P, _I32, _P, _P]),
    "burgers_tune_save": (_ST, [_P, ctypes.c_char_p]),
    "burgers_tune_load": (_ST, [_P, ctypes.c_char_p]),
}

class burgers_serve_cfg(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_active", ctypes.c_int64), ("hbm_budget", ctypes.c_int64),
                ("slice_steps", ctypes.c_int64), ("slice_timeout_s", ctypes.c_double)]


class burgers_request(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("bc", ctypes.c_int32), ("n", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("dx", ctypes.c_double), ("nu", ctypes.c_double),
                ("dt", ctypes.c_double), ("nsteps", ctypes.c_int64), ("u0_host", ctypes.c_void_p)]


class burgers_req_stats(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("slices", ctypes.c_int64),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class burgers_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("slices", ctypes.c_int64), ("active_max", ctypes.c_int64),
                ("pool_used_max", ctypes.c_int64), ("cell_updates", ctypes.c_double),
                ("pending", ctypes.c_int64), ("active", ctypes.c_int64),
                ("pool_bytes", ctypes.c_int64), ("pool_used", ctypes.c_int64),
                ("now_s", ctypes.c_double), ("t_enqueue_s", ctypes.c_double),
                ("t_slice_s", ctypes.c_double), ("t_copy_s", ctypes.c_double),
                ("t_gpu_s", ctypes.c_double), ("t_gpu_gap_s", ctypes.c_double)]


SIGNATURES.update({
    "burgers_serve_create": (_ST, [_P, _P, ctypes.POINTER(_P)]),
    "burgers_serve_submit": (_ST, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "burgers_serve_submit_timed": (_ST, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "burgers_serve_poll": (_ST, [_P, ctypes.c_uint64, _P, _P]),
    "burgers_serve_wait": (_ST, [_P, ctypes.c_uint64, _D, _P, _P]),
    "burgers_serve_cancel": (_ST, [_P, ctypes.c_uint64]),
    "burgers_serve_wait_any": (_ST, [_P, _D, ctypes.POINTER(ctypes.c_uint64)]),
    "burgers_serve_get_stats": (_ST, [_P, _P]),
    "burgers_serve_destroy": (_ST, [_P]),
})

_lock = threading.Lock()
_lib = None


class BurgersError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load() -> ctypes.CDLL:
    """Loads libburgers.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2601_12204_b300.build` (no CPU fallback exists)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def last_error() -> str:
    return load().burgers_last_error().decode(errors="replace")


def check(status: int, where: str) -> int:
    if status != BURGERS_OK:
        raise BurgersError(status, where, last_error())
    return status


def exported_symbols():
    """Names of SIGNATURES that the loaded library exports."""
    lib = load()
    out = []
    for name in SIGNATURES:
        try:
            getattr(lib, name)
            out.append(name)
        except AttributeError:
            pass
    return out
