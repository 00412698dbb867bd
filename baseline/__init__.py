"""Threaded CPU CSB SpMM baseline (the paper's CPU organisation of the product, Section 4.4).

A timing baseline for the GPU product: built with OpenMP, called from the bench and from its own
CPU test. It is neither the oracle nor a product path. ``csb_omp.c`` documents the layout.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csb_omp.c")
_LIB = os.path.join(_HERE, "libcsb_omp.so")
_lib = None


def build() -> str:
    """Compile with OpenMP; without it (no libgomp on the host) the same code runs on one thread,
    which ``max_threads()`` then reports."""
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O3", "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC]
        if subprocess.call(cmd[:2] + ["-fopenmp"] + cmd[2:]) != 0:
            subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.csb_build.restype = ctypes.c_void_p
        _lib.csb_build.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int]
        _lib.csb_free.argtypes = [ctypes.c_void_p]
        _lib.csb_spmm.restype = ctypes.c_int
        _lib.csb_spmm.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        _lib.csb_ntiles.restype = ctypes.c_int64
        _lib.csb_ntiles.argtypes = [ctypes.c_void_p]
        _lib.csb_max_threads.restype = ctypes.c_int
    return _lib


def max_threads() -> int:
    return int(lib().csb_max_threads())


class CsbMatrix:
    """Upper-triangle COO (row <= col) in b x b tiles with FP32 values."""

    def __init__(self, n, rows, cols, vals, b=256):
        L = lib()
        self._r = np.ascontiguousarray(rows, dtype=np.int64)
        c = np.ascontiguousarray(cols, dtype=np.int64)
        v = np.ascontiguousarray(vals, dtype=np.float64)
        self.n = int(n)
        self.nnz = len(self._r)
        self._h = L.csb_build(self.n, self.nnz, self._r.ctypes.data, c.ctypes.data, v.ctypes.data, b)
        if not self._h:
            raise ValueError("csb_build failed (bad entries, duplicates or no memory)")
        self.ntiles = int(L.csb_ntiles(self._h))
        del self._r

    def spmm(self, X, Y=None, threads=0):
        X = np.ascontiguousarray(X, dtype=np.float64)
        nb = X.shape[1]
        if Y is None:
            Y = np.empty_like(X)
        rc = lib().csb_spmm(self._h, X.ctypes.data, Y.ctypes.data, nb, threads)
        if rc != 0:
            raise RuntimeError(f"csb_spmm failed ({rc})")
        return Y

    def close(self):
        if self._h:
            lib().csb_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
