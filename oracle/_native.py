"""ctypes loader for oracle/native.c (test infrastructure only).

`build_native()` compiles the plain-C oracle routines with gcc into
oracle/_liboracle.so; `lib()` loads it (building on first use).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "native.c")
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build_native(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build_native()
            L = C.CDLL(_SO)
            i64, dp, vp = C.c_int64, C.POINTER(C.c_double), C.c_void_p
            L.or_chol_band.argtypes = [i64, i64, vp]
            L.or_chol_band.restype = C.c_int
            L.or_logdet_from_chol.argtypes = [i64, i64, vp]
            L.or_logdet_from_chol.restype = C.c_double
            L.or_lsolve_band.argtypes = [i64, i64, vp, i64, vp]
            L.or_lsolve_band.restype = None
            L.or_takahashi_diag.argtypes = [i64, i64, vp, vp]
            L.or_takahashi_diag.restype = None
            L.or_ldlt_band_z.argtypes = [i64, i64, vp]
            L.or_ldlt_band_z.restype = C.c_int
            L.or_fwd_quadform_z.argtypes = [i64, i64, vp, i64, vp, vp, vp]
            L.or_fwd_quadform_z.restype = None
            L.or_colour_greedy.argtypes = [i64, vp, vp, C.c_int, vp]
            L.or_colour_greedy.restype = C.c_int
            _lib = L
        return _lib


def ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)
