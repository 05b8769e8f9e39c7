"""Thin ctypes binding of libgbdcpu.so (include/gbdcpu.h): the paper's five-loop DGEMM on the
host cores (Section 3.1 and Section 4 of the paper).  It marshals arguments only; the
computation is the C library's.  Matrices are 1-D float64 numpy arrays in column-major
order with explicit leading dimensions, as in the BLAS statement (Section 2.1).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbdcpu.so")

_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libgbdcpu.so (building it in-tree with gcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            _build.build_cpu()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing and could not be built")
        lib = ctypes.CDLL(LIB_PATH)
        c, i64, d, i, vp = ctypes.c_char, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.gbd_cpu_dgemm.argtypes = [c, c, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64, i]
        lib.gbd_cpu_dgemm.restype = i
        ip = ctypes.POINTER(ctypes.c_int)
        lib.gbd_cpu_dgemm_blocking.argtypes = [ip, ip, ip, ip, ip]
        lib.gbd_cpu_dgemm_blocking.restype = None
        lib.gbd_cpu_max_threads.argtypes = []
        lib.gbd_cpu_max_threads.restype = i
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("expected a contiguous float64 numpy array")
    return a.ctypes.data


def gbd_cpu_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, threads=0) -> int:
    """C := alpha*op(A)*op(B) + beta*C in place on the host; returns the status (0, the BLAS
    index of the first invalid argument, or -1 when the packing buffers cannot be allocated)."""
    return load().gbd_cpu_dgemm(transa.encode(), transb.encode(), int(m), int(n), int(k), float(alpha), _ptr(A),
                                int(lda), _ptr(B), int(ldb), float(beta), _ptr(C), int(ldc), int(threads))


def blocking() -> dict:
    """The blocking parameters (mc, kc, nc, mr, nr) of gbd_cpu_dgemm."""
    v = [ctypes.c_int() for _ in range(5)]
    load().gbd_cpu_dgemm_blocking(*[ctypes.byref(x) for x in v])
    return dict(zip(("mc", "kc", "nc", "mr", "nr"), (x.value for x in v)))


def max_threads() -> int:
    return load().gbd_cpu_max_threads()
