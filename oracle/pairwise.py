"""ctypes loader for oracle/pairwise.c -- test infrastructure only.

``build()`` compiles the C file with gcc and OpenMP into oracle/_pairwise.so
(built on whichever machine runs it; the file is git-ignored).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pairwise.c")
_LIB = os.path.join(_HERE, "_pairwise.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_pairwise_matvec.argtypes = [ctypes.c_int64, dp, ctypes.c_double, dp, dp, dp]
        lib.oracle_pairwise_matvec.restype = ctypes.c_int
        lib.oracle_pairwise_rows.argtypes = [ctypes.c_int64, dp, ctypes.c_double, dp, dp,
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), dp]
        lib.oracle_pairwise_rows.restype = ctypes.c_int
        lib.oracle_field_points.argtypes = [ctypes.c_int64, dp, ctypes.c_double, dp, ctypes.c_int64, dp, dp]
        lib.oracle_field_points.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def matvec(r: np.ndarray, kd: float, beta: np.ndarray, P: np.ndarray, rows=None):
    """(A P) for all rows, or for the given row indices; P (N, 3) complex.

    Returns (Y, threads_used)."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.complex128)
    P = np.ascontiguousarray(P, dtype=np.complex128)
    n = r.shape[0]
    if rows is None:
        Y = np.empty((n, 3), dtype=np.complex128)
        nt = lib.oracle_pairwise_matvec(n, _dp(r), kd, _dp(beta), _dp(P), _dp(Y))
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        Y = np.empty((rows.size, 3), dtype=np.complex128)
        nt = lib.oracle_pairwise_rows(n, _dp(r), kd, _dp(beta), _dp(P), rows.size,
                                      rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(Y))
    return Y, nt


def scattered_field(r: np.ndarray, P: np.ndarray, x: np.ndarray, kd: float) -> np.ndarray:
    """E_sca at the points x (M, 3) from dipoles P (N, 3) at r (N, 3), the
    dipole on a point excluded (same definition as dda.scattered_field)."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.float64)
    E = np.empty((x.shape[0], 3), dtype=np.complex128)
    lib.oracle_field_points(r.shape[0], _dp(r), kd, _dp(P), x.shape[0], _dp(x), _dp(E))
    return E
