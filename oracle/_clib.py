"""Builds and loads the oracle's C deposit (oracle/deposit.c) with gcc.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "deposit.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_deposit.so")
_handle = None


def build(force: bool = False) -> str:
    """Compile deposit.c into a shared library next to it; returns the path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _handle
    if _handle is None:
        _handle = ctypes.CDLL(build())
        _handle.oracle_deposit_bspline.restype = None
        _handle.oracle_deposit_bspline.argtypes = [
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
    return _handle


def deposit_bspline(u: np.ndarray, q: np.ndarray, order: int, ng: int) -> np.ndarray:
    """u: (n,3) grid-unit positions, q: (n,nf) values -> (nf, ng, ng, ng) FP64 grids."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.ndim == 1:
        q = q[:, None]
    n, nf = q.shape
    assert u.shape == (n, 3)
    grids = np.zeros((nf, ng, ng, ng), dtype=np.float64)
    lib().oracle_deposit_bspline(n, u.ctypes.data, nf, q.ctypes.data, order, ng, grids.ctypes.data)
    return grids
