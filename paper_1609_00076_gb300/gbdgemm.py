"""Thin ctypes binding of libgbdgemm.so (include/gbdgemm.h).

Argument marshalling only: every step of every call runs in the CUDA library.
The functions keep the C names and argument order.  Matrix arguments accept a
torch tensor (its data_ptr() is passed), a raw integer device address, or None.
``stream`` accepts a torch.cuda.Stream, a raw cudaStream_t integer, or None for
torch's current stream.

There is no CPU fallback: if the shared library cannot be built or loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbdgemm.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "gbdgemm.h")

GBD_OK = 0
GBD_ERR_CUDA = -1
GBD_ERR_WORKSPACE = -2
GBD_ERR_TIMEOUT = -3
GBD_ERR_DEVICE = -4
GBD_ERR_LIMIT = -5
GBD_ERR_ARG = -6

_lock = threading.Lock()
_lib = None


class GbdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gbdgemm error {code}: {msg}")
        self.code = code


def load(build_if_missing: bool = True):
    """Load libgbdgemm.so (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise GbdError(GBD_ERR_CUDA, f"{LIB_PATH} is missing and could not be built")
        lib = ctypes.CDLL(LIB_PATH)
        _declare(lib)
        _lib = lib
        return lib


def _declare(lib):
    c, i64, d, i, vp, sz = (ctypes.c_char, ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                            ctypes.c_void_p, ctypes.c_size_t)
    lib.gbd_version.argtypes = []
    lib.gbd_version.restype = i
    lib.gbd_last_error.argtypes = []
    lib.gbd_last_error.restype = ctypes.c_char_p
    lib.gbd_dgemm.argtypes = [c, c, i64, i64, i64, d, vp, i64, vp, i64, d, vp, i64, vp]
    lib.gbd_dgemm.restype = i
    lib.gbd_check_device_error.argtypes = [vp]
    lib.gbd_check_device_error.restype = i
    for name, argt, rest in _EXTRA_DECLS:
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes = argt
            f.restype = rest


class GbdEmuInfo(ctypes.Structure):
    """Mirror of gbd_emu_info."""
    _fields_ = [("record_phases", ctypes.c_int), ("slices", ctypes.c_int), ("digit_bits", ctypes.c_int),
                ("products", ctypes.c_int), ("path", ctypes.c_int), ("exact", ctypes.c_int),
                ("rho", ctypes.c_double), ("gamma", ctypes.c_double), ("bound", ctypes.c_double),
                ("prep_ms", ctypes.c_double), ("gemm_ms", ctypes.c_double),
                ("recon_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_c, _i64, _d, _i, _vp, _sz = (ctypes.c_char, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_size_t)

GBD_MODE_NATIVE = 0
GBD_MODE_EMULATED = 1
GBD_MODE_MODULAR = 2

GBD_METHOD_NATIVE = 0
GBD_METHOD_SPLIT = 1
GBD_METHOD_MODULAR = 2
GBD_METHOD_AUTO = 3

GBD_PATH_NONE = 0
GBD_PATH_SPLIT = 1
GBD_PATH_MODULAR = 2
GBD_PATH_NATIVE = 3


class GbdProblem(ctypes.Structure):
    """Mirror of gbd_problem (one problem of a grouped call)."""
    _fields_ = [("transa", ctypes.c_char), ("transb", ctypes.c_char), ("ksplit", ctypes.c_uint8),
                ("reserved", ctypes.c_uint8), ("mode", ctypes.c_int32),
                ("slices", ctypes.c_int32), ("tile", ctypes.c_int32), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("k", ctypes.c_int64), ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("A", ctypes.c_void_p),
                ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("C", ctypes.c_void_p),
                ("ldc", ctypes.c_int64), ("tol", ctypes.c_double)]
# (name, argtypes, restype) of the entry points declared further down the header
_EXTRA_DECLS: list = [
    ("gbd_dgemm_emu_workspace_size", [_i64, _i64, _i64, _i], _sz),
    ("gbd_dgemm_emu", [_c, _c, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64, _i, _d, _vp, _sz,
                       ctypes.POINTER(GbdEmuInfo), _vp], _i),
    ("gbd_dgemm_emu_noalloc", [_c, _c, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64, _i, _d,
                               ctypes.POINTER(GbdEmuInfo), _vp], _i),
    ("gbd_dgemm_emu_mod_workspace_size", [_i64, _i64, _i64, _i], _sz),
    ("gbd_abs_product_lower_bound_workspace_size", [_i64, _i64, _i64], _sz),
    ("gbd_abs_product_lower_bound", [_c, _c, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i, _vp, _sz, _vp],
     _i),
    ("gbd_dgemm_emu_mod_moduli", [_i, _i64, ctypes.POINTER(ctypes.c_int)], _i),
    ("gbd_dgemm_emu_mod", [_c, _c, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64, _i, _d, _vp, _sz,
                           ctypes.POINTER(GbdEmuInfo), _vp], _i),
    ("gbd_dsyrk_workspace_size", [_i64, _i64, _i], _sz),
    ("gbd_dtrmm_workspace_size", [_c, _i64, _i64, _i], _sz),
    ("gbd_dtrsm_workspace_size", [_c, _i64, _i64, _i], _sz),
    ("gbd_dsyrk", [_c, _c, _i64, _i64, _d, _vp, _i64, _d, _vp, _i64, _i, _d, _vp, _sz, _vp], _i),
    ("gbd_dtrmm", [_c, _c, _c, _c, _i64, _i64, _d, _vp, _i64, _vp, _i64, _i, _d, _vp, _sz, _vp], _i),
    ("gbd_dtrsm", [_c, _c, _c, _c, _i64, _i64, _d, _vp, _i64, _vp, _i64, _i, _d, _vp, _sz, _vp], _i),
    ("gbd_dgemm_emu_host_buffer_size", [_c, _c, _i64, _i64, _i64, _i], _sz),
    ("gbd_dgemm_emu_mod_host_buffer_size", [_c, _c, _i64, _i64, _i64, _i], _sz),
    ("gbd_dgemm_emu_mod_host", [_c, _c, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64, _i, _d, _vp, _sz,
                                ctypes.POINTER(GbdEmuInfo), _vp], _i),
    ("gbd_dgemm_emu_host", [_c, _c, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64, _i, _d, _vp, _sz,
                            ctypes.POINTER(GbdEmuInfo), _vp], _i),
    ("gbd_watchdog_selftest", [_i, _vp], _i),
    ("gbd_fp64_mma_probe", [_i64, ctypes.POINTER(_d), _vp], _i),
    ("gbd_create", [ctypes.POINTER(_vp), _i], _i),
    ("gbd_destroy", [_vp], None),
    ("gbd_workspace_size", [_vp, _i, _i64, _i64, _i64, ctypes.POINTER(_sz)], _i),
    ("gbd_ctx_dgemm", [_vp, _i, _c, _c, _i64, _i64, _i64, _d, _vp, _i64, _vp, _i64, _d, _vp, _i64, _d,
                       ctypes.POINTER(GbdEmuInfo), _vp], _i),
    ("gbd_ctx_dgemm_grouped", [_vp, _vp, _i, _vp, _vp], _i),
    ("gbd_sync_error", [_vp, _vp], _i),
    ("gbd_ctx_pool_bytes", [_vp], _sz),
    ("gbd_dgemm_grouped_workspace_size", [_vp, _i], _sz),
    ("gbd_grouped_plan_create", [_vp, _i, _vp, _sz, _vp, _vp, ctypes.POINTER(_vp)], _i),
    ("gbd_grouped_plan_run", [_vp, _vp], _i),
    ("gbd_grouped_plan_destroy", [_vp], None),
    ("gbd_dgemm_grouped", [_vp, _i, _vp, _sz, _vp, _vp], _i),
]


def header_functions() -> list[str]:
    """Names of the functions declared in include/gbdgemm.h."""
    with open(HEADER_PATH) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbd_[a-z0-9_]+)\s*\(", text)))


def _addr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch tensor (device or host)
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):  # numpy array (host)
        return int(x.ctypes.data)
    raise TypeError(f"expected a device tensor or address, got {type(x)!r}")


def _stream(s) -> int | None:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    raise TypeError(f"expected a stream, got {type(s)!r}")


def _t(ch: str) -> bytes:
    b = ch.encode() if isinstance(ch, str) else bytes(ch)
    if len(b) != 1:
        raise ValueError("trans must be one character")
    return b


def gbd_version() -> int:
    return load().gbd_version()


def gbd_last_error() -> str:
    return load().gbd_last_error().decode(errors="replace")


def check(rc: int) -> int:
    """Raise GbdError for a non-zero status, with the library's message."""
    if rc != 0:
        raise GbdError(rc, gbd_last_error())
    return rc


def gbd_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None) -> int:
    """C := alpha*op(A)*op(B) + beta*C on the native FP64 MMA path; returns the status."""
    return load().gbd_dgemm(_t(transa), _t(transb), int(m), int(n), int(k), float(alpha), _addr(A),
                            int(lda), _addr(B), int(ldb), float(beta), _addr(C), int(ldc),
                            _stream(stream))


def gbd_dgemm_emu_workspace_size(m, n, k, slices=0) -> int:
    """Device workspace bytes of gbd_dgemm_emu (slices 0 = automatic, sized for 9)."""
    return int(load().gbd_dgemm_emu_workspace_size(int(m), int(n), int(k), int(slices)))


def gbd_dgemm_emu(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, tol, workspace,
                  workspace_bytes, info=None, stream=None) -> int:
    """C := alpha*op(A)*op(B) + beta*C by split emulation on the BF16 tensor cores; returns the
    status.  ``info`` may be a GbdEmuInfo to receive the report."""
    return load().gbd_dgemm_emu(_t(transa), _t(transb), int(m), int(n), int(k), float(alpha), _addr(A),
                                int(lda), _addr(B), int(ldb), float(beta), _addr(C), int(ldc), int(slices),
                                float(tol), _addr(workspace), int(workspace_bytes),
                                ctypes.byref(info) if info is not None else None, _stream(stream))


def gbd_dgemm_emu_noalloc(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, tol, info=None,
                          stream=None) -> int:
    """gbd_dgemm_emu without a caller workspace (built-in 64 MiB scratch); returns the status."""
    return load().gbd_dgemm_emu_noalloc(_t(transa), _t(transb), int(m), int(n), int(k), float(alpha), _addr(A),
                                        int(lda), _addr(B), int(ldb), float(beta), _addr(C), int(ldc), int(slices),
                                        float(tol), ctypes.byref(info) if info is not None else None, _stream(stream))


def gbd_dgemm_emu_mod_workspace_size(m, n, k, bits=0) -> int:
    """Device workspace bytes of gbd_dgemm_emu_mod (bits 0 = automatic, sized for 16 moduli)."""
    return int(load().gbd_dgemm_emu_mod_workspace_size(int(m), int(n), int(k), int(bits)))


def gbd_dgemm_emu_mod_moduli(bits, k) -> list:
    """The moduli of the modular emulation for `bits` integer bits at inner dimension k ([] if 16
    are not enough)."""
    out = (ctypes.c_int * 16)()
    n = int(load().gbd_dgemm_emu_mod_moduli(int(bits), int(k), out))
    return [int(out[i]) for i in range(n)]


def gbd_dgemm_emu_mod(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, bits, tol, workspace,
                      workspace_bytes, info=None, stream=None) -> int:
    """C := alpha*op(A)*op(B) + beta*C by the modular emulation (residue products and the Chinese
    remainder theorem) on the BF16 tensor cores; returns the status."""
    return load().gbd_dgemm_emu_mod(_t(transa), _t(transb), int(m), int(n), int(k), float(alpha), _addr(A),
                                    int(lda), _addr(B), int(ldb), float(beta), _addr(C), int(ldc), int(bits),
                                    float(tol), _addr(workspace), int(workspace_bytes),
                                    ctypes.byref(info) if info is not None else None, _stream(stream))


def gbd_abs_product_lower_bound_workspace_size(m, n, k) -> int:
    """Device workspace bytes of gbd_abs_product_lower_bound."""
    return int(load().gbd_abs_product_lower_bound_workspace_size(int(m), int(n), int(k)))


def gbd_abs_product_lower_bound(transa, transb, m, n, k, A, lda, B, ldb, L, ldl, fp8, workspace, workspace_bytes,
                                stream=None) -> int:
    """L := a guaranteed lower bound of |op(A)||op(B)| (the certification product, BF16 or FP8 E5M2
    planes); returns the status."""
    return load().gbd_abs_product_lower_bound(_t(transa), _t(transb), int(m), int(n), int(k), _addr(A), int(lda),
                                              _addr(B), int(ldb), _addr(L), int(ldl), int(fp8), _addr(workspace),
                                              int(workspace_bytes), _stream(stream))


def gbd_dsyrk_workspace_size(n, k, mode) -> int:
    """Device workspace bytes of gbd_dsyrk."""
    return int(load().gbd_dsyrk_workspace_size(int(n), int(k), int(mode)))


def gbd_dtrmm_workspace_size(side, m, n, mode) -> int:
    """Device workspace bytes of gbd_dtrmm."""
    return int(load().gbd_dtrmm_workspace_size(_t(side), int(m), int(n), int(mode)))


def gbd_dtrsm_workspace_size(side, m, n, mode) -> int:
    """Device workspace bytes of gbd_dtrsm."""
    return int(load().gbd_dtrsm_workspace_size(_t(side), int(m), int(n), int(mode)))


def gbd_dsyrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, mode, tol, workspace, workspace_bytes,
              stream=None) -> int:
    """C := alpha op(A) op(A)^T + beta C on one triangle (GEMM-based); returns the status."""
    return load().gbd_dsyrk(_t(uplo), _t(trans), int(n), int(k), float(alpha), _addr(A), int(lda), float(beta),
                            _addr(C), int(ldc), int(mode), float(tol), _addr(workspace), int(workspace_bytes),
                            _stream(stream))


def gbd_dtrmm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, mode, tol, workspace, workspace_bytes,
              stream=None) -> int:
    """B := alpha op(A) B or alpha B op(A), A triangular (GEMM-based); returns the status."""
    return load().gbd_dtrmm(_t(side), _t(uplo), _t(transa), _t(diag), int(m), int(n), float(alpha), _addr(A),
                            int(lda), _addr(B), int(ldb), int(mode), float(tol), _addr(workspace),
                            int(workspace_bytes), _stream(stream))


def gbd_dtrsm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, mode, tol, workspace, workspace_bytes,
              stream=None) -> int:
    """B := X with op(A) X = alpha B or X op(A) = alpha B (GEMM-based); returns the status."""
    return load().gbd_dtrsm(_t(side), _t(uplo), _t(transa), _t(diag), int(m), int(n), float(alpha), _addr(A),
                            int(lda), _addr(B), int(ldb), int(mode), float(tol), _addr(workspace),
                            int(workspace_bytes), _stream(stream))


def gbd_dgemm_emu_host_buffer_size(transa, transb, m, n, k, slices=0) -> int:
    """Device buffer bytes of gbd_dgemm_emu_host (packed A, B, C and the workspace)."""
    return int(load().gbd_dgemm_emu_host_buffer_size(_t(transa), _t(transb), int(m), int(n), int(k), int(slices)))


def gbd_dgemm_emu_host(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, tol, buffer,
                       buffer_bytes, info=None, stream=None) -> int:
    """gbd_dgemm_emu with A, B and C in host memory (numpy arrays or host tensors; page-locked
    for asynchronous transfers) and a caller-owned device buffer; returns the status."""
    return load().gbd_dgemm_emu_host(_t(transa), _t(transb), int(m), int(n), int(k), float(alpha), _addr(A),
                                     int(lda), _addr(B), int(ldb), float(beta), _addr(C), int(ldc), int(slices),
                                     float(tol), _addr(buffer), int(buffer_bytes),
                                     ctypes.byref(info) if info is not None else None, _stream(stream))


def gbd_dgemm_emu_mod_host_buffer_size(transa, transb, m, n, k, bits=0) -> int:
    """Device buffer bytes of gbd_dgemm_emu_mod_host (packed A, B, C and the modular workspace)."""
    return int(load().gbd_dgemm_emu_mod_host_buffer_size(_t(transa), _t(transb), int(m), int(n), int(k),
                                                         int(bits)))


def gbd_dgemm_emu_mod_host(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, bits, tol, buffer,
                           buffer_bytes, info=None, stream=None) -> int:
    """gbd_dgemm_emu_mod with A, B and C in host memory and a caller-owned device buffer."""
    return load().gbd_dgemm_emu_mod_host(_t(transa), _t(transb), int(m), int(n), int(k), float(alpha), _addr(A),
                                         int(lda), _addr(B), int(ldb), float(beta), _addr(C), int(ldc), int(bits),
                                         float(tol), _addr(buffer), int(buffer_bytes),
                                         ctypes.byref(info) if info is not None else None, _stream(stream))


def problem_array(problems) -> ctypes.Array:
    """A ctypes array of GbdProblem from GbdProblem objects or dicts of its fields."""
    arr = (GbdProblem * max(1, len(problems)))()
    for i, p in enumerate(problems):
        if isinstance(p, GbdProblem):
            arr[i] = p
            continue
        q = GbdProblem()
        for key, val in p.items():
            if key in ("A", "B", "C"):
                val = _addr(val)
            elif key in ("transa", "transb"):
                val = _t(val)
            setattr(q, key, val)
        arr[i] = q
    return arr


def gbd_dgemm_grouped_workspace_size(problems) -> int:
    arr = problems if isinstance(problems, ctypes.Array) else problem_array(problems)
    return int(load().gbd_dgemm_grouped_workspace_size(ctypes.cast(arr, _vp), len(arr) if problems else 0))


def gbd_grouped_plan_create(problems, workspace, workspace_bytes, slices_used=None, stream=None):
    """Returns (status, plan handle); slices_used may be a ctypes int array of len(problems)."""
    arr = problems if isinstance(problems, ctypes.Array) else problem_array(problems)
    plan = _vp()
    rc = load().gbd_grouped_plan_create(ctypes.cast(arr, _vp), len(problems), _addr(workspace), int(workspace_bytes),
                                        ctypes.cast(slices_used, _vp) if slices_used is not None else None,
                                        _stream(stream), ctypes.byref(plan))
    return rc, plan


def gbd_grouped_plan_run(plan, stream=None) -> int:
    return load().gbd_grouped_plan_run(plan, _stream(stream))


def gbd_grouped_plan_destroy(plan) -> None:
    load().gbd_grouped_plan_destroy(plan)


def gbd_dgemm_grouped(problems, workspace, workspace_bytes, slices_used=None, stream=None) -> int:
    arr = problems if isinstance(problems, ctypes.Array) else problem_array(problems)
    return load().gbd_dgemm_grouped(ctypes.cast(arr, _vp), len(problems), _addr(workspace), int(workspace_bytes),
                                    ctypes.cast(slices_used, _vp) if slices_used is not None else None,
                                    _stream(stream))


def gbd_create(device: int = 0):
    """Returns (status, context handle)."""
    ctx = _vp()
    rc = load().gbd_create(ctypes.byref(ctx), int(device))
    return rc, ctx


def gbd_destroy(ctx) -> None:
    load().gbd_destroy(ctx)


def gbd_workspace_size(ctx, method, m, n, k):
    """Returns (status, bytes) of the workspace `method` takes (ctx may be None)."""
    out = _sz(0)
    rc = load().gbd_workspace_size(ctx, int(method), int(m), int(n), int(k), ctypes.byref(out))
    return rc, int(out.value)


def gbd_ctx_dgemm(ctx, method, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tol=0.0, info=None,
                  stream=None) -> int:
    """C := alpha*op(A)*op(B) + beta*C by `method` with the context's workspace pool."""
    return load().gbd_ctx_dgemm(ctx, int(method), _t(transa), _t(transb), int(m), int(n), int(k), float(alpha),
                                _addr(A), int(lda), _addr(B), int(ldb), float(beta), _addr(C), int(ldc), float(tol),
                                ctypes.byref(info) if info is not None else None, _stream(stream))


def gbd_ctx_dgemm_grouped(ctx, problems, slices_used=None, stream=None) -> int:
    arr = problems if isinstance(problems, ctypes.Array) else problem_array(problems)
    return load().gbd_ctx_dgemm_grouped(ctx, ctypes.cast(arr, _vp), len(problems),
                                        ctypes.cast(slices_used, _vp) if slices_used is not None else None,
                                        _stream(stream))


def gbd_sync_error(ctx, stream=None) -> int:
    return load().gbd_sync_error(ctx, _stream(stream))


def gbd_ctx_pool_bytes(ctx) -> int:
    return int(load().gbd_ctx_pool_bytes(ctx))


def gbd_fp64_mma_probe(iters: int = 20000, stream=None):
    """Returns (status, measured FP64 tensor-core TFLOP/s)."""
    out = _d(0.0)
    rc = load().gbd_fp64_mma_probe(int(iters), ctypes.byref(out), _stream(stream))
    return rc, float(out.value)


def gbd_watchdog_selftest(limit_ms: int, stream=None) -> int:
    return load().gbd_watchdog_selftest(int(limit_ms), _stream(stream))


def gbd_check_device_error(stream=None) -> int:
    return load().gbd_check_device_error(_stream(stream))


# ---------------------------------------------------------------------------
# torch helpers for the column-major layout (Section 2.1 of the paper)
# ---------------------------------------------------------------------------
def colmajor_view(buf, rows: int, cols: int, ld: int):
    """rows x cols column-major view (strides (1, ld)) of a flat tensor of ld*cols elements."""
    return buf[: ld * cols].view(cols, ld)[:, :rows].t() if cols else buf[:0].view(0, 0)


def to_device(np_buf, device="cuda"):
    """Copy a flat numpy float64 buffer to a flat device tensor."""
    import torch
    return torch.from_numpy(np_buf).to(device)
