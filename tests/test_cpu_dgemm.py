"""Parity of the host five-loop DGEMM (libgbdcpu.so, the paper's Section 3.1 and Section 4)
with the oracle.

The operation is the dgemm of Section 1.2 with column-major storage (Section 2.1).  Each
element is summed over k in increasing order in blocks of kc, with alpha applied per block
and beta once, so the error is within (k + 2) u G, G = |alpha||op(A)||op(B)| + |beta||C0|
(the standard bound of a recursively summed dot product plus the two scalings).  The shapes
cross every blocking boundary: mr, nr, mc, kc and nc.
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import cpu_blas, synth


def _stored(t, rows, cols):
    return (cols, rows) if t == "T" else (rows, cols)


def _problem(ta, tb, m, n, k, seed, pads=(0, 0, 0), kind="uniform"):
    ra, ca = _stored(ta, m, k)
    rb, cb = _stored(tb, k, n)
    lda, ldb, ldc = max(1, ra + pads[0]), max(1, rb + pads[1]), max(1, m + pads[2])
    A = synth.matrix(kind, ra, ca, lda, seed)
    B = synth.matrix(kind, rb, cb, ldb, seed + 1)
    C = synth.matrix(kind, m, n, ldc, seed + 2)
    return A, lda, B, ldb, C, ldc


def _check(oracle_mod, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, threads=0):
    C = C0.copy()
    assert cpu_blas.gbd_cpu_dgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, threads) == 0
    ref = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    got = synth.view(C, m, n, ldc).flatten(order="F")
    msg = first_mismatch(got, ref, (k + 2) * U * G, m)
    assert msg is None, msg
    # padding rows of C untouched
    full = C.reshape(n, ldc) if ldc * n == C.size else None
    if full is not None and ldc > m:
        assert np.array_equal(full[:, m:], C0.reshape(n, ldc)[:, m:], equal_nan=True)
    return C


def test_exports_every_declared_symbol():
    import ctypes
    import os
    import re
    header = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gbdcpu.h")
    text = re.sub(r"/\*.*?\*/", "", open(header).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(gbd_[a-z0-9_]+)\s*\(", text)))
    assert "gbd_cpu_dgemm" in names
    cpu_blas.load()
    raw = ctypes.CDLL(cpu_blas.LIB_PATH)
    assert not [x for x in names if not hasattr(raw, x)]


def test_blocking():
    b = cpu_blas.blocking()
    assert b == {"mc": 128, "kc": 256, "nc": 3072, "mr": 8, "nr": 6}
    assert cpu_blas.max_threads() >= 1


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 3), (9, 13, 257), (129, 7, 300), (200, 150, 520)])
def test_parity_transposes_and_fringes(oracle_mod, ta, tb, m, n, k):
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, 100 + m + n + k, pads=(2, 1, 3))
    _check(oracle_mod, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc)


def test_parity_across_column_blocks(oracle_mod):
    # n > nc: two passes of loop 5, the second one partial
    m, n, k = 37, 3100, 20
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, 7, pads=(0, 3, 1))
    _check(oracle_mod, "N", "T", m, n, k, -0.75, A, lda, B, ldb, 2.0, C, ldc)


def test_same_bits_for_any_thread_count(oracle_mod):
    m, n, k = 300, 70, 600
    A, lda, B, ldb, C, ldc = _problem("T", "N", m, n, k, 9, pads=(1, 0, 2))
    outs = [_check(oracle_mod, "T", "N", m, n, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, threads=t) for t in (1, 3, 0)]
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint64), outs[0].view(np.uint64))


def test_integer_inputs_exact():
    m, n, k = 70, 90, 530
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, 11, kind="int8")
    Cw = C.copy()
    assert cpu_blas.gbd_cpu_dgemm("N", "N", m, n, k, 2.0, A, lda, B, ldb, -1.0, Cw, ldc) == 0
    Ai = synth.view(A, m, k, lda).astype(np.int64)
    Bi = synth.view(B, k, n, ldb).astype(np.int64)
    want = 2 * (Ai @ Bi) - synth.view(C, m, n, ldc).astype(np.int64)
    assert np.array_equal(synth.view(Cw, m, n, ldc), want.astype(np.float64))


def test_beta_zero_does_not_read_c(oracle_mod):
    m, n, k = 20, 30, 40
    A, lda, B, ldb, _, ldc = _problem("N", "N", m, n, k, 13)
    C = np.full(ldc * n, np.nan)
    assert cpu_blas.gbd_cpu_dgemm("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc) == 0
    ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, np.zeros(ldc * n), ldc)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, np.zeros(ldc * n), ldc)
    assert first_mismatch(synth.view(C, m, n, ldc).flatten(order="F"), ref, (k + 2) * U * G, m) is None


def test_quick_returns():
    m, n, k = 6, 5, 4
    nanA = np.full(m * k, np.nan)
    nanB = np.full(k * n, np.nan)
    C0 = synth.matrix("uniform", m, n, m, 17, pad=0.0)
    # alpha == 0: C := beta C, A and B not read
    C = C0.copy()
    assert cpu_blas.gbd_cpu_dgemm("N", "N", m, n, k, 0.0, nanA, m, nanB, k, 0.5, C, m) == 0
    assert np.array_equal(C, 0.5 * C0)
    # k == 0 with beta == 0: zeros, C not read
    C = np.full(m * n, np.nan)
    assert cpu_blas.gbd_cpu_dgemm("N", "N", m, n, 0, 1.0, nanA, m, nanB, 1, 0.0, C, m) == 0
    assert np.array_equal(C, np.zeros(m * n))
    # (alpha == 0 or k == 0) with beta == 1, and m == 0 or n == 0: nothing touched
    C = np.full(m * n, np.nan)
    assert cpu_blas.gbd_cpu_dgemm("N", "N", m, n, 0, 1.0, nanA, m, nanB, 1, 1.0, C, m) == 0
    assert np.isnan(C).all()
    assert cpu_blas.gbd_cpu_dgemm("N", "N", 0, n, k, 1.0, nanA, 1, nanB, k, 0.0, C, 1) == 0
    assert cpu_blas.gbd_cpu_dgemm("N", "N", m, 0, k, 1.0, nanA, m, nanB, k, 0.0, C, m) == 0
    assert np.isnan(C).all()


@pytest.mark.parametrize("args,code", [
    (("X", "N", 2, 2, 2, 2, 2, 2), 1), (("N", "X", 2, 2, 2, 2, 2, 2), 2), (("N", "N", -1, 2, 2, 2, 2, 2), 3),
    (("N", "N", 2, -1, 2, 2, 2, 2), 4), (("N", "N", 2, 2, -1, 2, 2, 2), 5), (("N", "N", 3, 2, 2, 2, 2, 3), 8),
    (("T", "N", 2, 2, 3, 2, 3, 2), 8), (("N", "N", 2, 2, 3, 2, 2, 2), 10), (("N", "T", 2, 3, 2, 2, 2, 2), 10),
    (("N", "N", 3, 2, 2, 3, 2, 2), 13)])
def test_argument_codes(args, code):
    ta, tb, m, n, k, lda, ldb, ldc = args
    buf = np.zeros(64)
    assert cpu_blas.gbd_cpu_dgemm(ta, tb, m, n, k, 1.0, buf, lda, buf, ldb, 0.0, buf, ldc) == code
