"""ctypes declarations of the C ABI in include/lbcuboid.h (argument marshalling only).

The library is loaded from this package directory (built in-tree by build.py).
There is no fallback: if liblbcuboid.so is missing or cannot be loaded, every
entry point raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbcuboid.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EUNSTABLE, LB_ETIMEOUT, LB_ESTATE = range(7)
LB_F64, LB_F32, LB_F32_SHIFTED, LB_F16_SHIFTED, LB_BF16_SHIFTED = range(5)
LB_CORR_NONE, LB_CORR_LOWMACH, LB_CORR_LOCAL, LB_CORR_FULL = range(4)
LB_WALL_X, LB_WALL_Y, LB_WALL_Z = 1, 2, 4

STATUS_NAMES = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_EUNSTABLE",
                5: "LB_ETIMEOUT", 6: "LB_ESTATE"}


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class lb_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("r_y", ctypes.c_double), ("r_z", ctypes.c_double),
        ("nu", ctypes.c_double), ("zeta", ctypes.c_double), ("cs2", ctypes.c_double),
        ("storage", ctypes.c_int), ("corr", ctypes.c_int), ("wall_mask", ctypes.c_uint),
        ("force", ctypes.c_double * 3), ("lid_u", ctypes.c_double), ("stream", ctypes.c_void_p),
        ("rounding", ctypes.c_int), ("rounding_seed", ctypes.c_uint), ("kernel", ctypes.c_int),
        ("model", ctypes.c_int), ("subdomains", ctypes.c_int),
    ]


# name -> (restype, argtypes); every symbol declared in include/lbcuboid.h
_P = ctypes.c_void_p
_CTX = ctypes.c_void_p
SIGNATURES = {
    "lb_config_default": (None, [ctypes.POINTER(lb_config), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "lb_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    "lb_create_ex": (ctypes.c_int, [ctypes.POINTER(lb_config), ctypes.POINTER(ctypes.c_void_p)]),
    "lb_destroy": (None, [_CTX]),
    "lb_real_size": (ctypes.c_int, [_CTX]),
    "lb_num_nodes": (ctypes.c_size_t, [_CTX]),
    "lb_get_params": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double)]),
    "lb_init": (ctypes.c_int, [_CTX, _P, _P]),
    "lb_set_force_field": (ctypes.c_int, [_CTX, _P]),
    "lb_step": (ctypes.c_int, [_CTX, ctypes.c_int]),
    "lb_moments": (ctypes.c_int, [_CTX, _P, _P]),
    "lb_reduce": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double)]),
    "lb_get_populations": (ctypes.c_int, [_CTX, _P]),
    "lb_set_populations": (ctypes.c_int, [_CTX, _P]),
    "lb_state_bytes": (ctypes.c_size_t, [_CTX]),
    "lb_get_state": (ctypes.c_int, [_CTX, _P]),
    "lb_set_state": (ctypes.c_int, [_CTX, _P, ctypes.c_longlong]),
    "lb_time_step": (ctypes.c_longlong, [_CTX]),
    "lb_set_force": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double)]),
    "lb_set_rates": (ctypes.c_int, [_CTX, ctypes.c_double, ctypes.c_double]),
    "lb_set_lid": (ctypes.c_int, [_CTX, ctypes.c_double]),
    "lb_objective_ke": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double)]),
    "lb_adjoint_ke": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "lb_adjoint": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    "lb_collide_vjp": (ctypes.c_int, [_CTX, ctypes.c_longlong, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "lb_reduce_populations_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong, ctypes.c_double,
                                                      ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                                      ctypes.POINTER(ctypes.c_double), _P]),
    "lb_step_kernel": (ctypes.c_char_p, [_CTX]),
    "lb_selftest_bounded_wait": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "lb_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load liblbcuboid.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2107_14774_gb300.build.build() "
                              "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int) -> None:
    if status != LB_OK:
        raise LBError(status, load().lb_last_error().decode())
