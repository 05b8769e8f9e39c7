"""Parity of the native FP64-MMA DGEMM (gbd_dgemm) with the CPU oracle.

Bar: bit-exact on small-integer inputs (every partial sum is an exact integer),
otherwise the componentwise bound |C - C_oracle| <= 2 k u G with
G = |alpha||op(A)||op(B)| + |beta||C0| and u = 2^-53.  Every call runs on device
buffers surrounded by NaN guard bands, and the leading-dimension padding of C
holds NaN sentinels: both must come back untouched.
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, DeviceBuf, first_mismatch, padding_intact
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def _stored(trans, rows, cols):
    return (cols, rows) if trans in "TtCc" else (rows, cols)


def run_native(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, offsets=(0, 0, 0), stream=None):
    import torch
    dA = DeviceBuf(A, offset=offsets[0])
    dB = DeviceBuf(B, offset=offsets[1])
    dC = DeviceBuf(C, offset=offsets[2])
    torch.cuda.synchronize()  # the copies above ran on torch's stream; `stream` may be another
    rc = gbdgemm.gbd_dgemm(ta, tb, m, n, k, alpha, dA.ptr, lda, dB.ptr, ldb, beta, dC.ptr, ldc, stream=stream)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    assert dA.guards_intact() and dB.guards_intact() and dC.guards_intact()
    assert np.array_equal(dA.host().view(np.uint64), A.view(np.uint64))  # inputs untouched
    out = dC.host()
    assert padding_intact(out, m, n, ldc)
    return out


def _problem(ta, tb, m, n, k, kind, seed, pads=(0, 0, 0), e=0):
    ra, ca = _stored(ta, m, k)
    rb, cb = _stored(tb, k, n)
    lda, ldb, ldc = ra + pads[0], rb + pads[1], m + pads[2]
    A = synth.matrix(kind, ra, ca, lda, seed, e=e)
    B = synth.matrix(kind, rb, cb, ldb, seed + 1, e=e)
    C = synth.matrix("uniform" if kind != "int8" else "int8", m, n, ldc, seed + 2)
    return A, lda, B, ldb, C, ldc


def _compact(C, m, n, ldc):
    return np.ascontiguousarray(synth.view(C, m, n, ldc)).flatten(order="F")


def check_against_oracle(oracle_mod, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, out, exact=False,
                         rows=None):
    ref = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, rows=rows)
    got = _compact(out, m, n, ldc)
    nr = m
    if rows is not None:
        got = got.reshape(n, m)[:, rows].flatten()
        nr = len(rows)
    if exact:
        msg = first_mismatch(got, ref, None, nr)
    else:
        G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, rows=rows)
        msg = first_mismatch(got, ref, 2 * k * U * G, nr)
    assert msg is None, msg


# --- 256^3, N,N, alpha=1, beta=0 (uniform and small integers) ---
def test_square_256_uniform(oracle_mod):
    m = n = k = 256
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "uniform", synth.seed_for(0))
    out = run_native("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc)
    check_against_oracle(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out)


def test_square_256_integers_bit_exact(oracle_mod):
    m = n = k = 256
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "int8", synth.seed_for(0, 1))
    out = run_native("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc)
    check_against_oracle(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out, exact=True)


# --- 1000 x 1200 x 800, four transposes, ld + 8, alpha 1.5, beta -0.5 ---
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_padded_ld_all_transposes(oracle_mod, ta, tb):
    m, n, k = 1000, 1200, 800
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "uniform", synth.seed_for(1), pads=(8, 8, 8))
    out = run_native(ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc)
    check_against_oracle(oracle_mod, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, out)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_integers_bit_exact_all_transposes(oracle_mod, ta, tb):
    m, n, k = 300, 270, 513
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "int8", 77, pads=(2, 4, 6))
    out = run_native(ta, tb, m, n, k, 2.0, A, lda, B, ldb, -1.0, C, ldc)
    check_against_oracle(oracle_mod, ta, tb, m, n, k, 2.0, A, lda, B, ldb, -1.0, C, ldc, out, exact=True)


# --- fringes: every residue class against the 16-deep k tile and both CTA tiles ---
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 9, 15), (33, 65, 16), (63, 31, 17), (65, 100, 47),
                                   (129, 1, 200), (1, 257, 3)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T"), ("T", "N")])
def test_fringes_small_tiles(oracle_mod, m, n, k, ta, tb):
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "uniform", m * 7 + n * 13 + k, pads=(2, 0, 4))
    out = run_native(ta, tb, m, n, k, -1.25, A, lda, B, ldb, 0.5, C, ldc)
    check_against_oracle(oracle_mod, ta, tb, m, n, k, -1.25, A, lda, B, ldb, 0.5, C, ldc, out)


@pytest.mark.parametrize("m,n,k", [(1001, 999, 37), (830, 1030, 16), (1024, 960, 1)])
@pytest.mark.parametrize("ta,tb", [("N", "T"), ("T", "N")])
def test_fringes_large_tiles(oracle_mod, m, n, k, ta, tb):
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "uniform", m + n + k, pads=(0, 6, 2))
    out = run_native(ta, tb, m, n, k, 1.0, A, lda, B, ldb, 1.0, C, ldc)
    check_against_oracle(oracle_mod, ta, tb, m, n, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, out)


# --- the non-TMA loader: odd leading dimensions and 8-byte (not 16-byte) aligned bases ---
@pytest.mark.parametrize("pads,offsets", [((1, 3, 1), (0, 0, 0)), ((0, 0, 0), (1, 1, 1)), ((2, 2, 2), (1, 0, 1))])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
def test_unaligned_fallback(oracle_mod, pads, offsets, ta, tb):
    m, n, k = 130, 97, 75
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "uniform", 5, pads=pads)
    out = run_native(ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, offsets=offsets)
    check_against_oracle(oracle_mod, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, out)


def test_paper_leading_dimension_example(oracle_mod):
    """Section 1.2: a 2 x 2 sub-matrix passed as an interior pointer with lda = 3."""
    arr = np.array([1.1, 2.1, 3.1, 1.2, 2.2, 3.2, 1.3, 2.3, 3.3])
    dArr = DeviceBuf(arr)
    B = np.array([1.0, 0.0, 0.0, 1.0])
    dB = DeviceBuf(B)
    dC = DeviceBuf(None, n=4)
    rc = gbdgemm.gbd_dgemm("N", "N", 2, 2, 2, 1.0, dArr.ptr + 3 * 8, 3, dB.ptr, 2, 0.0, dC.ptr, 2, stream=None)
    assert rc == 0, gbdgemm.gbd_last_error()
    assert np.array_equal(dC.host(), np.array([1.2, 2.2, 1.3, 2.3]))
    # the sub-matrix times itself, against the oracle given the same interior pointer
    rc = gbdgemm.gbd_dgemm("N", "N", 2, 2, 2, 1.0, dArr.ptr + 24, 3, dArr.ptr + 24, 3, 0.0, dC.ptr, 2, stream=None)
    assert rc == 0
    ref = oracle_mod.dgemm_rows("N", "N", 2, 2, 2, 1.0, arr[3:].copy(), 3, arr[3:].copy(), 3, 0.0, None, 2)
    got = dC.host()
    G = oracle_mod.abs_bound_rows("N", "N", 2, 2, 2, 1.0, arr[3:].copy(), 3, arr[3:].copy(), 3, 0.0, None, 2)
    assert first_mismatch(got, ref, 4 * U * G, 2) is None
    assert dArr.guards_intact() and dC.guards_intact()


# --- BLAS quick returns ---
def test_quick_returns():
    m, n, k = 40, 30, 20
    nanA = np.full(m * k, np.nan)
    nanB = np.full(k * n, np.nan)
    C = synth.uniform_pm1(1, m * n)
    out = run_native("N", "N", m, n, k, 0.0, nanA, m, nanB, k, -2.0, C, m)
    assert np.array_equal(out, -2.0 * C)   # alpha == 0: A, B not read
    out = run_native("N", "N", m, n, 0, 1.0, nanA, m, nanB, 1, 0.5, C, m)
    assert np.array_equal(out, 0.5 * C)    # k == 0
    out = run_native("N", "N", m, n, k, 0.0, nanA, m, nanB, k, 1.0, C, m)
    assert np.array_equal(out, C)          # alpha == 0, beta == 1: untouched
    A = synth.uniform_pm1(2, m * k)
    B = synth.uniform_pm1(3, k * n)
    out = run_native("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, np.full(m * n, np.nan), m)
    assert np.isfinite(out).all()          # beta == 0: C not read


def test_deterministic_and_stream():
    import torch
    m, n, k = 700, 500, 900
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, "uniform", 3)
    s = torch.cuda.Stream()
    o1 = run_native("N", "T", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, stream=s)
    o2 = run_native("N", "T", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc)
    assert np.array_equal(o1.view(np.uint64), o2.view(np.uint64))


# --- 8192^3 (native leg) at the bench's launch, sampled rows ---
@pytest.mark.parametrize("e", [0, 8, 32])
def test_large_square_sampled_rows(oracle_mod, e):
    import torch
    m = n = k = 8192
    A = synth.matrix("scaled", m, k, m, synth.seed_for(2, e), e=e, pad=0.0)
    B = synth.matrix("scaled", k, n, k, synth.seed_for(2, e) + 1, e=e, pad=0.0)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.empty(m * n, dtype=torch.float64, device="cuda")
    rc = gbdgemm.gbd_dgemm("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    rows = sorted(set(int(x) for x in synth.splitmix64(synth.seed_for(2, e) + 7, 12) % m))
    got = dC.view(n, m)[:, rows].t().cpu().numpy().flatten(order="F")
    ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, rows=rows)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, rows=rows)
    msg = first_mismatch(got, ref, 2 * k * U * G, len(rows))
    assert msg is None, msg
