"""Build and load the C half of the oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fkski_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def lib_path() -> str:
    return _SO


def build(force: bool = False) -> str:
    """Compile fkski_oracle.c with gcc (-ffp-contract=off keeps the key arithmetic as written;
    -fopenmp for the precompute's cell-slab threads)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class OrGrid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("M", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
                ("h", ctypes.c_double * 3)]


def or_grid(grid) -> OrGrid:
    g = OrGrid()
    g.d = grid.d
    for k in range(3):
        g.M[k] = int(grid.M[k]) if k < grid.d else 1
        g.lo[k] = float(grid.lo[k]) if k < grid.d else 0.0
        g.h[k] = float(grid.h[k]) if k < grid.d else 1.0
    return g


def get():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        L.or_cell_key_f32.argtypes = [ctypes.c_float, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_double)]
        L.or_cell_key_f64.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_double)]
        L.or_keys_u.argtypes = [ctypes.c_double]
        L.or_keys_u.restype = ctypes.c_double
        L.or_keys_weights.argtypes = [ctypes.c_double, P]
        L.or_rademacher.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        L.or_rademacher.restype = ctypes.c_double
        L.or_rademacher_fill.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, P]
        L.or_keys.argtypes = [ctypes.POINTER(OrGrid), P, ctypes.c_int, ctypes.c_int64, P, P]
        L.or_w_rows.argtypes = [ctypes.POINTER(OrGrid), P, ctypes.c_int, ctypes.c_int64, P, P]
        L.or_precompute.argtypes = [ctypes.POINTER(OrGrid), P, ctypes.c_int, P, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_uint64, P, P, P, P, P, P, P]
        L.or_predict.argtypes = [ctypes.POINTER(OrGrid), P, P, ctypes.c_int, ctypes.c_int64, P]
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_set_threads.restype = None
        L.or_max_threads.argtypes = []
        L.or_max_threads.restype = ctypes.c_int
        for f in ("or_keys", "or_w_rows", "or_precompute", "or_predict", "or_cell_key_f32",
                  "or_cell_key_f64"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None
