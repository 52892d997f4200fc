"""ctypes loader for the oracle's plain-C quadrature (oracle/quad.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  build() compiles quad.c with gcc
(-O2, OpenMP, no -march flags so it builds the same on x86-64 and aarch64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "quad.c")
_LIB = os.path.join(_HERE, "_quad.so")
_lib = None

NANG, NRAD, PIECE = 6, 5, 1.0


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        _lib = L
        set_rule(NANG, NRAD, PIECE)
        for name in ("oq_h0", "oq_h0dot", "oq_q0"):
            getattr(L, name).restype = ctypes.c_double
            getattr(L, name).argtypes = [ctypes.c_double, ctypes.c_double]
    return _lib


_keep = []


def set_rule(nang: int, nrad: int, piece: float):
    """Select the inner-rule orders (default 6, 5, 1.0; larger values are a refinement)."""
    ax, aw = np.polynomial.legendre.leggauss(nang)
    rx, rw = np.polynomial.legendre.leggauss(nrad)
    _keep[:] = [np.ascontiguousarray(a) for a in (ax, aw, rx, rw)]
    lib().oq_set_rules(ctypes.c_int(nang), P(_keep[0]), P(_keep[1]), ctypes.c_int(nrad), P(_keep[2]), P(_keep[3]),
                       ctypes.c_double(piece))


def set_time_order(p: int):
    """Temporal basis of the retarded matrices: 1 the paper's hat / C1-quadratic pair, 2 the shifted
    quadratic Lagrange interpolator with its compatible q (quad.c)."""
    assert p in (1, 2)
    lib().oq_set_time_order(ctypes.c_int(p))


def P(a: np.ndarray):
    """Pointer to a C-contiguous numpy array."""
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def I(x):
    return ctypes.c_int(int(x))


def D(x):
    return ctypes.c_double(float(x))


def triangle_moments(x, v0, v1, v2, kind: int, p1: float = 0.0, p2: float = 0.0, brk=(), coplanar=False):
    """Polar-rule moments over one triangle: (m0, m1) of kernel `kind` about x (see quad.c)."""
    out = np.zeros(4)
    b = np.ascontiguousarray(np.asarray(brk, dtype=np.float64))
    args = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (x, v0, v1, v2)]
    lib().oq_triangle_moments(*(P(a) for a in args), P(b) if b.size else None, I(b.size), I(int(coplanar)),
                              I(kind), D(p1), D(p2), P(out))
    return out[0], out[1:]
