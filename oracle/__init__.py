"""CPU oracle for C := alpha*op(A)*op(B) + beta*C (paper Section 1.2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The product path
(``paper_1609_00076_gb300``) never imports it, and this package never imports
the product: the two share no code.

Contents
--------
* ``dgemm_rows`` / ``dgemm``: the plain definition, element by element, with
  compensated (Dot2, Ogita-Rump-Oishi 2005) accumulation, in C (oracle.c).
* ``abs_bound_rows``: G = |alpha||op(A)||op(B)| + |beta||C0|, the magnitude in the
  componentwise bound |C - C_exact| <= 2 k 2^-53 G.
* ``ozaki_dgemm_rows``: a plain CPU model of the split emulation (ozaki_model.c),
  same digits, same level order, same segment order as the GPU emulation but
  written independently (floating-point digit recursion instead of bit fields).
* ``ozmod_dgemm_rows``: a plain CPU model of the modular emulation (Ozaki scheme II,
  ozaki_mod_model.c): rounded scaled integers and their exact 128-bit product, where
  the GPU path goes through residues and the Chinese remainder theorem.
* ``certify``: the certified precision choice of both emulations (certify.c): the
  smallest slice count / integer bit count whose a-priori truncation bound stays within
  the componentwise target on every element, from the exact |op(A)||op(B)|, or the
  exactness width when every scaled entry is an integer.
* ``dsyrk`` / ``dtrmm`` / ``dtrsm``: the GEMM-based level-3 operations by their plain
  definitions (level3.c): Dot2 inner products on the referenced triangle, and
  substitution with Dot2 numerators for the triangular solve.

Matrices are passed as 1-D float64 numpy arrays in column-major order with an
explicit leading dimension, exactly as in the BLAS statement (Section 2.1:
element (i, j) lives at index j*ld + i).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["oracle.c", "ozaki_model.c", "ozaki_mod_model.c", "level3.c", "certify.c"]
_lib = None


class CertChoice(ctypes.Structure):
    """Mirror of oracle_cert_t (certify.c)."""
    _fields_ = [("t_cert", ctypes.c_int), ("t_exact", ctypes.c_int), ("t", ctypes.c_int),
                ("moduli", ctypes.c_int), ("s_cert", ctypes.c_int), ("s_exact", ctypes.c_int),
                ("s", ctypes.c_int), ("pad", ctypes.c_int), ("rho", ctypes.c_double),
                ("gamma", ctypes.c_double), ("alpha2", ctypes.c_double), ("beta2", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no value-changing FP optimisation)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        lib_mtime = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_mtime for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-pthread", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    d, i64, c, i = ctypes.c_double, ctypes.c_int64, ctypes.c_char, ctypes.c_int
    vp = ctypes.c_void_p
    lib.oracle_dgemm_rows.argtypes = [c, c, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64, vp,
                                      i64, vp, i64, i]
    lib.oracle_dgemm_rows.restype = i
    lib.oracle_abs_bound_rows.argtypes = lib.oracle_dgemm_rows.argtypes
    lib.oracle_abs_bound_rows.restype = i
    lib.oracle_dgemm.argtypes = [c, c, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64, i]
    lib.oracle_dgemm.restype = i
    lib.oracle_ozaki_dgemm_rows.argtypes = [c, c, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64,
                                            i, i, i64, vp, i64, vp, i64, i]
    lib.oracle_ozaki_dgemm_rows.restype = i
    lib.oracle_ozaki_exponent.argtypes = [d]
    lib.oracle_ozaki_exponent.restype = i
    lib.oracle_ozaki_split.argtypes = [d, i, i, i, vp]
    lib.oracle_ozaki_split.restype = None
    lib.oracle_ozmod_dgemm_rows.argtypes = [c, c, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64,
                                            i, vp, i64, vp, i64, i]
    lib.oracle_ozmod_dgemm_rows.restype = i
    lib.oracle_ozmod_i128_to_double.argtypes = [i64, ctypes.c_uint64]
    lib.oracle_ozmod_i128_to_double.restype = d
    lib.oracle_dsyrk.argtypes = [c, c, i64, i64, d, vp, i64, d, vp, i64, i]
    lib.oracle_dsyrk.restype = i
    lib.oracle_dtrmm.argtypes = [c, c, c, c, i64, i64, d, vp, i64, vp, i64, i]
    lib.oracle_dtrmm.restype = i
    lib.oracle_dtrsm.argtypes = lib.oracle_dtrmm.argtypes
    lib.oracle_dtrsm.restype = i
    lib.oracle_certify.argtypes = [c, c, i64, i64, i64, vp, i64, vp, i64, d, vp, i64, i,
                                   ctypes.POINTER(CertChoice)]
    lib.oracle_certify.restype = i
    lib.oracle_cert_moduli.argtypes = [i, i64]
    lib.oracle_cert_moduli.restype = i
    lib.oracle_cert_moduli_cs.argtypes = [i, i64, ctypes.c_double, ctypes.c_double]
    lib.oracle_cert_moduli_cs.restype = i
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = i
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data


def _as_f64(a):
    if a is None:
        return None
    a = np.asarray(a)
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("oracle matrices are contiguous float64 1-D buffers")
    return a


def num_threads() -> int:
    return _load().oracle_num_threads()


def _rows_arg(rows, m):
    if rows is None:
        return None, m
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    return r, int(r.size)


def dgemm_rows(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, rows=None,
               nthreads=0):
    """Rows ``rows`` (default: all) of alpha*op(A)*op(B) + beta*C0 as an
    (nrows x n) column-major buffer (leading dimension nrows).  C0 is not modified."""
    lib = _load()
    r, nr = _rows_arg(rows, m)
    out = np.empty(max(1, nr) * max(1, n), dtype=np.float64)
    rc = lib.oracle_dgemm_rows(transa.encode(), transb.encode(), m, n, k, float(alpha),
                               _ptr(_as_f64(A)), lda, _ptr(_as_f64(B)), ldb, float(beta),
                               _ptr(_as_f64(C0)), ldc, _ptr(r), nr, out.ctypes.data, max(1, nr),
                               int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_dgemm_rows: invalid argument {rc}")
    return out[: nr * n]


def dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=0):
    """In place, the exact dgemm argument list: C is overwritten.  Returns the
    BLAS status (0, or the index of the first invalid argument)."""
    lib = _load()
    return lib.oracle_dgemm(transa.encode(), transb.encode(), m, n, k, float(alpha),
                            _ptr(_as_f64(A)), lda, _ptr(_as_f64(B)), ldb, float(beta),
                            _ptr(_as_f64(C)), ldc, int(nthreads))


def abs_bound_rows(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, rows=None,
                   nthreads=0):
    """Rows of |alpha||op(A)||op(B)| + |beta||C0| (same layout as dgemm_rows)."""
    lib = _load()
    r, nr = _rows_arg(rows, m)
    out = np.empty(max(1, nr) * max(1, n), dtype=np.float64)
    rc = lib.oracle_abs_bound_rows(transa.encode(), transb.encode(), m, n, k, float(alpha),
                                   _ptr(_as_f64(A)), lda, _ptr(_as_f64(B)), ldb, float(beta),
                                   _ptr(_as_f64(C0)), ldc, _ptr(r), nr, out.ctypes.data,
                                   max(1, nr), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_abs_bound_rows: invalid argument {rc}")
    return out[: nr * n]


def ozaki_dgemm_rows(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, slices,
                     bits=7, kseg=8192, rows=None, nthreads=0):
    """Rows of the split emulation (model of the GPU path) with ``slices`` digits of
    ``bits`` bits per operand and level sums over segments of ``kseg`` indices."""
    lib = _load()
    r, nr = _rows_arg(rows, m)
    out = np.empty(max(1, nr) * max(1, n), dtype=np.float64)
    rc = lib.oracle_ozaki_dgemm_rows(transa.encode(), transb.encode(), m, n, k, float(alpha),
                                     _ptr(_as_f64(A)), lda, _ptr(_as_f64(B)), ldb, float(beta),
                                     _ptr(_as_f64(C0)), ldc, int(slices), int(bits), int(kseg),
                                     _ptr(r), nr, out.ctypes.data, max(1, nr), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_ozaki_dgemm_rows: status {rc}")
    return out[: nr * n]


def ozmod_dgemm_rows(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, bits, rows=None,
                     nthreads=0):
    """Rows of the modular emulation (model of the GPU path) with ``bits`` integer bits."""
    lib = _load()
    r, nr = _rows_arg(rows, m)
    out = np.empty(max(1, nr) * max(1, n), dtype=np.float64)
    rc = lib.oracle_ozmod_dgemm_rows(transa.encode(), transb.encode(), m, n, k, float(alpha),
                                     _ptr(_as_f64(A)), lda, _ptr(_as_f64(B)), ldb, float(beta),
                                     _ptr(_as_f64(C0)), ldc, int(bits), _ptr(r), nr, out.ctypes.data,
                                     max(1, nr), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_ozmod_dgemm_rows: status {rc}")
    return out[: nr * n]


def ozmod_i128_to_double(v: int) -> float:
    """The model's conversion of a 128-bit integer to double."""
    u = v & ((1 << 128) - 1)
    hi = u >> 64
    if hi >= 1 << 63:
        hi -= 1 << 64
    return _load().oracle_ozmod_i128_to_double(hi, u & ((1 << 64) - 1))


def dsyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, nthreads=0):
    """In place on the `uplo` triangle of C: C := alpha op(A) op(A)^T + beta C.  Returns the
    BLAS status."""
    return _load().oracle_dsyrk(uplo.encode(), trans.encode(), n, k, float(alpha), _ptr(_as_f64(A)), lda,
                                float(beta), _ptr(_as_f64(C)), ldc, int(nthreads))


def dtrmm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, nthreads=0):
    """In place: B := alpha op(A) B (side 'L') or alpha B op(A) (side 'R'), A triangular."""
    return _load().oracle_dtrmm(side.encode(), uplo.encode(), transa.encode(), diag.encode(), m, n,
                                float(alpha), _ptr(_as_f64(A)), lda, _ptr(_as_f64(B)), ldb, int(nthreads))


def dtrsm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, nthreads=0):
    """In place: B := X with op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R')."""
    return _load().oracle_dtrsm(side.encode(), uplo.encode(), transa.encode(), diag.encode(), m, n,
                                float(alpha), _ptr(_as_f64(A)), lda, _ptr(_as_f64(B)), ldb, int(nthreads))


def ozaki_exponent(x: float) -> int:
    return _load().oracle_ozaki_exponent(float(x))


def ozaki_split(x: float, sigma: int, slices: int, bits: int = 7) -> list[int]:
    out = np.zeros(16, dtype=np.int32)
    _load().oracle_ozaki_split(float(x), int(sigma), int(slices), int(bits), out.ctypes.data)
    return [int(v) for v in out[:slices]]


def certify(transa, transb, m, n, k, A, lda, B, ldb, tol=0.0, rows=None, nthreads=0) -> dict:
    """The certified precision choice of both emulations (certify.c) for rows ``rows``
    (default: all) of op(A) against every column of op(B).  Keys: t_cert, t_exact, t
    (63: infeasible), moduli (0: infeasible), s_cert, s_exact, s (10: infeasible), rho,
    gamma, alpha2, beta2."""
    lib = _load()
    r, nr = _rows_arg(rows, m)
    out = CertChoice()
    rc = lib.oracle_certify(transa.encode(), transb.encode(), m, n, k, _ptr(_as_f64(A)), lda,
                            _ptr(_as_f64(B)), ldb, float(tol), _ptr(r), nr, int(nthreads),
                            ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"oracle_certify: status {rc}")
    return {f: getattr(out, f) for f, _ in CertChoice._fields_ if f != "pad"}


def cert_moduli(t: int, k: int) -> int:
    """Fewest leading moduli whose product exceeds 2 k 2^(2t) (0: more than 16)."""
    return _load().oracle_cert_moduli(int(t), int(k))


def cert_moduli_cs(t: int, k: int, alpha2: float, beta2: float) -> int:
    """Fewest leading moduli whose product exceeds twice min(k 2^(2t),
    (2^t alpha + sqrt(k)/2)(2^t beta + sqrt(k)/2)) (0: more than 16), alpha^2 and beta^2 the
    largest scaled square sums of the rows of op(A) and the columns of op(B)."""
    return _load().oracle_cert_moduli_cs(int(t), int(k), float(alpha2), float(beta2))
