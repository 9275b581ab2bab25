"""ctypes wrapper of the plain-C cyclic Jacobi eigensolver (oracle/jacobi.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).

§III, step 1: all eigenvalues and eigenvectors of the symmetric H. The result
is sorted ascending, V[:, i] is the unit eigenvector of w[i].
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi.c")
_LIB = os.path.join(_HERE, "_jacobi.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile oracle/jacobi.c with gcc (OpenMP) into oracle/_jacobi.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC,
               "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB)
            f = lib.oracle_jacobi_eigh
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_double)]
            _lib = lib
    return _lib


def jacobi_eigh(H, max_sweeps: int = 60, return_info: bool = False):
    """Eigen-decomposition of symmetric H by cyclic Jacobi; ascending order."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    if H.shape != (n, n):
        raise ValueError("H must be square")
    if n == 0:
        w, V = np.zeros(0), np.zeros((0, 0))
        return (w, V, {"sweeps": 0, "off": 0.0}) if return_info else (w, V)
    A = np.ascontiguousarray(H.copy())
    w = np.empty(n, dtype=np.float64)
    V = np.empty((n, n), dtype=np.float64)
    sweeps = ctypes.c_int(0)
    off = ctypes.c_double(0.0)
    rc = _load().oracle_jacobi_eigh(n, A.ctypes.data, w.ctypes.data, V.ctypes.data,
                                    max_sweeps, ctypes.byref(sweeps), ctypes.byref(off))
    if rc != 0:
        raise RuntimeError(f"oracle_jacobi_eigh failed ({rc})")
    order = np.argsort(w, kind="stable")
    w = w[order]
    V = V[:, order]
    if return_info:
        return w, V, {"sweeps": sweeps.value, "off": off.value}
    return w, V
