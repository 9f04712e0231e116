"""ctypes access to oracle.c (plain C, FP64).  Test infrastructure only.

Built with gcc (OpenMP) into oracle/_build/liboracle.so by build().
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    # -ffp-contract=off: no fused multiply-add, every operation rounds as written
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.fo_spmm.argtypes = [ctypes.c_int64, vp, vp, vp, ctypes.c_int, vp]
            lib.fo_spmm_rows.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int64, vp, vp]
            lib.fo_jacobi.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_double, ctypes.c_int]
            lib.fo_jacobi.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def spmm(rowptr: np.ndarray, colidx: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = A X with A the 0/1 pattern of (rowptr, colidx); FP64 accumulate (Section 3.3).

    X may be float32 or float64; float32 values are widened exactly to float64 first.
    """
    lib = _load()
    n = rowptr.shape[0] - 1
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    b = X.shape[1]
    assert X.shape[0] == n and 1 <= b <= 64
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    Y = np.empty((n, b), np.float64)
    lib.fo_spmm(n, _ptr(rp), _ptr(ci), _ptr(X), b, _ptr(Y))
    return Y


def spmm_rows(rowptr: np.ndarray, colidx: np.ndarray, X: np.ndarray, rows) -> np.ndarray:
    """(A X)[rows, :], computed row by row as in spmm()."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    b = X.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    Y = np.empty((rows.size, b), np.float64)
    lib.fo_spmm_rows(_ptr(rp), _ptr(ci), _ptr(X), b, rows.size, _ptr(rows), _ptr(Y))
    return Y


def jacobi(T: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Eigen-decomposition of a symmetric T by cyclic Jacobi (Golub & Van Loan Sec. 8.5).

    Returns (theta, Y) with T Y = Y diag(theta), Y orthogonal; theta in Jacobi's order.
    """
    lib = _load()
    A = np.array(T, dtype=np.float64, order="C", copy=True)
    m = A.shape[0]
    assert A.shape == (m, m)
    ev = np.empty(m)
    V = np.empty((m, m))
    sweeps = lib.fo_jacobi(m, _ptr(A), _ptr(ev), _ptr(V), tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge")
    return ev, V
