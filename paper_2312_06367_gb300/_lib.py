"""ctypes binding of libtdcfie.so (argument marshalling only; all compute runs in the library).

There is no CPU fallback: if the shared library is missing or fails to load, load() raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdcfie.so")

FP64, FP32, BF16X3, FP16X3 = 0, 1, 2, 3
SOLVE_DIRECT, SOLVE_GMRES = 0, 1
GUESS_ZERO, GUESS_PREV, GUESS_MLP, GUESS_EXTRAP, GUESS_MLP_EXTRAP = 0, 1, 2, 3, 4
MLP_NPARAM = 4801
STATUS = {0: "OK", -1: "E_ARG", -2: "E_MESH", -3: "E_OOM", -4: "E_CUDA", -5: "E_NOCONV", -6: "E_TIMEOUT",
          -7: "E_NONFINITE", -8: "E_STATE", -9: "E_UNSUPPORTED"}


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("solver", ctypes.c_int), ("gmres_tol", ctypes.c_double),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int), ("guess", ctypes.c_int),
                ("max_rhs", ctypes.c_int64), ("stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("time_order", ctypes.c_int)]


class PlaneWaves(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int64), ("k_hat", ctypes.c_void_p), ("pol", ctypes.c_void_p),
                ("amp", ctypes.c_void_p), ("t0", ctypes.c_void_p), ("width", ctypes.c_void_p)]


class TdcfieError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes) of every entry point declared in include/tdcfie.h
_P, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
SIGNATURES = [
    ("tdcfie_default_opts", None, [_P]),
    ("tdcfie_create", _I, [_P, _I64, _P, _I64, _D, _I64, _D, _P, _P]),
    ("tdcfie_assemble", _I, [_P]),
    ("tdcfie_set_excitation", _I, [_P, _P]),
    ("tdcfie_step", _I, [_P, _I64, _P]),
    ("tdcfie_march", _I, [_P, _P, _P, _I]),
    ("tdcfie_step_y", _I, [_P, _I64, _P, _P]),
    ("tdcfie_gmres_stats", _I, [_P, _P, _P, _P, _P]),
    ("tdcfie_info", _I, [_P, _P, _P, _P, _P, _P, _P]),
    ("tdcfie_topology", _I, [_P, _P, _P, _P]),
    ("tdcfie_bc_table", _I, [_P, _P, _P, _P, _P, _P, _P]),
    ("tdcfie_get_matrix", _I, [_P, _I, _I64, _P]),
    ("tdcfie_last_timing", _I, [_P, _P, _P, _P, _P]),
    ("tdcfie_assembly_timing", _I, [_P, _P]),
    ("tdcfie_block_gemv", _I, [_I, _P, _I64, _I64, _P, _I64, _P, _P]),
    ("tdcfie_block_gemv_noalloc", _I, [_I, _P, _I64, _I64, _P, _I64, _P, _P]),
    ("tdcfie_tc_gemm", _I, [_I, _P, _I64, _I64, _I64, _P, _I64, _P, _P]),
    ("tdcfie_mlp_grad", _I, [_P, _P, _P, _I64, _P, _P, _P]),
    ("tdcfie_mlp_train", _I, [_P, _P, _P, _I64, _I, _I64, ctypes.c_float, ctypes.c_uint64, _P, _P]),
    ("tdcfie_mlp_predict", _I, [_P, _P, _I64, _P, _P]),
    ("tdcfie_mlp_samples", _I, [_I, _I, _P, _I64, _I64, _I64, _P, _P, _P]),
    ("tdcfie_mlp_load", _I, [_P, _P]),
    ("tdcfie_set_solver", _I, [_P, _I, _I, _D]),
    ("tdcfie_replan", _I, [_P, _I, _I64]),
    ("tdcfie_set_history_form", _I, [_P, _I]),
    ("tdcfie_far_field", _I, [_P, _P, _I64, _D, _P, _I64, _P]),
    ("tdcfie_set_formulation", _I, [_P, _I]),
    ("tdcfie_history_stats", _I, [_P, _P, _P, _P, _P]),
    ("tdcfie_batch_create", _I, [_P, _I64, _P]),
    ("tdcfie_batch_step", _I, [_P, _I64, _P]),
    ("tdcfie_batch_tune", _I, [_P, _I64, _P]),
    ("tdcfie_batch_timing", _I, [_P, _P, _P]),
    ("tdcfie_batch_destroy", _I, [_P]),
    ("tdcfie_release_assembly", _I, [_P]),
    ("tdcfie_destroy", _I, [_P]),
    ("tdcfie_last_error", ctypes.c_char_p, [_P]),
]


def load():
    """Load the in-tree shared library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def check(status: int, handle=None):
    if status != 0:
        msg = load().tdcfie_last_error(handle).decode(errors="replace")
        raise TdcfieError(status, msg)


def default_opts() -> Opts:
    o = Opts()
    load().tdcfie_default_opts(ctypes.byref(o))
    return o
