"""Pins of the CPU model of the split emulation (oracle/ozaki_model.c).

The model restates the error-free splitting of Ozaki, Ogita, Oishi and Rump
(Numer. Algorithms 59, 2012) in fixed-point digit form.  These tests tie it to
exact arithmetic: digit bounds and reconstruction, closed forms, exact integer
products, a rational a-priori error bound, and the plain Dot2 oracle.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import synth


def _exact_product(ta, tb, m, n, k, A, lda, B, ldb):
    def a(i, p):
        return Fraction(float(A[i * lda + p] if ta else A[p * lda + i]))

    def b(p, j):
        return Fraction(float(B[p * ldb + j] if tb else B[j * ldb + p]))

    return [[sum((a(i, p) * b(p, j) for p in range(k)), Fraction(0)) for j in range(n)] for i in range(m)]


def test_exponent_convention(oracle_mod):
    # x = f * 2^e with 0.5 <= |f| < 1
    assert oracle_mod.ozaki_exponent(1.0) == 1
    assert oracle_mod.ozaki_exponent(0.5) == 0
    assert oracle_mod.ozaki_exponent(0.75) == 0
    assert oracle_mod.ozaki_exponent(-8.0) == 4
    assert oracle_mod.ozaki_exponent(7.999) == 3
    assert oracle_mod.ozaki_exponent(0.0) == 0
    assert oracle_mod.ozaki_exponent(5e-324) == -1073
    assert oracle_mod.ozaki_exponent(1.7976931348623157e308) == 1024


@pytest.mark.parametrize("bits", [7, 8, 5])
def test_split_digits_and_reconstruction(oracle_mod, bits):
    xs = list(synth.scaled_uniform(5, 200, 30)) + [0.0, 1.0 - 2.0 ** -53, -0.5, 2.0 ** -1074]
    for x in xs:
        sigma = oracle_mod.ozaki_exponent(x)
        for s in (1, 2, 4, 7):
            if s * bits > 63:
                continue
            d = oracle_mod.ozaki_split(x, sigma, s, bits)
            assert all(abs(v) <= 2 ** bits - 1 for v in d)
            assert all(v == 0 or (v > 0) == (x > 0) for v in d)  # truncation keeps the sign
            recon = sum((Fraction(v) * Fraction(2) ** (sigma - (t + 1) * bits) for t, v in enumerate(d)), Fraction(0))
            err = Fraction(x) - recon
            # truncation toward zero: remainder has the sign of x and is below one unit of the last digit
            assert abs(err) < Fraction(2) ** (sigma - s * bits)
            assert err == 0 or (err > 0) == (x > 0)
        # 8 digits of 7 bits cover the 53-bit significand when x sets the row exponent
        if bits == 7 and x != 0 and abs(x) >= 2.0 ** -1000:
            d = oracle_mod.ozaki_split(x, sigma, 8, 7)
            recon = sum((Fraction(v) * Fraction(2) ** (sigma - (t + 1) * 7) for t, v in enumerate(d)), Fraction(0))
            assert recon == Fraction(x)


@pytest.mark.parametrize("slices", [1, 3, 7])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_integer_inputs_exact(oracle_mod, slices, ta, tb):
    m, n, k = 21, 18, 257
    ra, ca = (k, m) if ta == "T" else (m, k)
    rb, cb = (n, k) if tb == "T" else (k, n)
    A = synth.matrix("int8", ra, ca, ra + 3, 1)
    B = synth.matrix("int8", rb, cb, rb, 2)
    C0 = synth.matrix("int8", m, n, m + 1, 3)
    Ai = synth.view(A, ra, ca, ra + 3).astype(np.int64)
    Bi = synth.view(B, rb, cb, rb).astype(np.int64)
    Ai = Ai.T if ta == "T" else Ai
    Bi = Bi.T if tb == "T" else Bi
    Ci = synth.view(C0, m, n, m + 1).astype(np.int64)
    out = oracle_mod.ozaki_dgemm_rows(ta, tb, m, n, k, 2.0, A, ra + 3, B, rb, -1.0, C0, m + 1, slices)
    assert np.array_equal(out.reshape(n, m).T, (2 * (Ai @ Bi) - Ci).astype(np.float64))


def test_all_ones_closed_form(oracle_mod):
    m, n, k = 5, 7, 1000
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.5, np.ones(m * k), m, np.ones(k * n), k, 0.0,
                                      None, m, 4)
    assert np.all(out == 1.5 * k)


def _apriori_bound(oracle_mod, ta, tb, m, n, k, alpha, A, lda, B, ldb, s, bits):
    """|alpha| 2^(sigma_i+tau_j-s*b) (mu_i + nu_j + (s-1)(1+2^-b) k), exact rationals."""
    def a(i, p):
        return float(A[i * lda + p] if ta else A[p * lda + i])

    def b(p, j):
        return float(B[p * ldb + j] if tb else B[j * ldb + p])

    sig = [max([oracle_mod.ozaki_exponent(a(i, p)) for p in range(k) if a(i, p) != 0] or [0]) for i in range(m)]
    tau = [max([oracle_mod.ozaki_exponent(b(p, j)) for p in range(k) if b(p, j) != 0] or [0]) for j in range(n)]
    mu = [sum(abs(Fraction(a(i, p))) for p in range(k)) / Fraction(2) ** sig[i] for i in range(m)]
    nu = [sum(abs(Fraction(b(p, j))) for p in range(k)) / Fraction(2) ** tau[j] for j in range(n)]
    c = Fraction(s - 1) * (1 + Fraction(1, 2 ** bits)) * k
    return [[abs(Fraction(alpha)) * Fraction(2) ** (sig[i] + tau[j] - s * bits) * (mu[i] + nu[j] + c)
             for j in range(n)] for i in range(m)]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("slices", [2, 3, 5])
def test_truncation_bound_vs_rational(oracle_mod, seed, slices):
    m, n, k = 4, 3, 9
    e = 12
    A = synth.matrix("scaled", m, k, m, 100 + seed, e=e)
    B = synth.matrix("scaled", k, n, k, 200 + seed, e=e)
    alpha = 1.25
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, alpha, A, m, B, k, 0.0, None, m, slices)
    exact = _exact_product(False, False, m, n, k, A, m, B, k)
    bound = _apriori_bound(oracle_mod, False, False, m, n, k, alpha, A, m, B, k, slices, 7)
    for i in range(m):
        for j in range(n):
            ex = Fraction(alpha) * exact[i][j]
            err = abs(Fraction(out[j * m + i]) - ex)
            # + the FP64 rounding of the (s+1) fused updates
            tol = bound[i][j] + Fraction((slices + 2) * U) * (abs(ex) + bound[i][j])
            assert err <= tol, (i, j, float(err), float(tol))


def test_level_scale_is_pinned(oracle_mod):
    # One non-zero digit per operand at known positions: a_00 = 2^-7 (digit 1 of
    # slice 2 when sigma = 1 from a_01 = 1), b_00 = 1 (slice 1).  The product lands in
    # level g = 3 and must come back exactly as 2^-7.
    A = np.array([2.0 ** -7, 1.0])  # row 0 of op(A) = [2^-7, 1] stored 1 x 2 (lda = 1)
    B = np.array([1.0, 0.0])        # column 0 of op(B) = [1, 0]
    out = oracle_mod.ozaki_dgemm_rows("N", "N", 1, 1, 2, 1.0, A, 1, B, 2, 0.0, None, 1, 2)
    assert out[0] == 2.0 ** -7
    # with a single slice the level-3 product is dropped: the result is the truncated 0
    out = oracle_mod.ozaki_dgemm_rows("N", "N", 1, 1, 2, 1.0, A, 1, B, 2, 0.0, None, 1, 1)
    assert out[0] == 0.0


@pytest.mark.parametrize("e", [0, 8, 32])
def test_nine_slices_within_fp64_bound(oracle_mod, e):
    m, n, k = 48, 40, 384
    A = synth.matrix("scaled", m, k, m + 2, 300 + e, e=e)
    B = synth.matrix("scaled", k, n, k, 400 + e, e=e)
    C0 = synth.matrix("uniform", m, n, m, 500 + e)
    ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.5, A, m + 2, B, k, -0.5, C0, m)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.5, A, m + 2, B, k, -0.5, C0, m)
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.5, A, m + 2, B, k, -0.5, C0, m, 9)
    assert first_mismatch(out, ref, 2 * k * U * G, m) is None


def test_segment_order_only_changes_rounding(oracle_mod):
    m, n, k = 9, 8, 300
    A = synth.matrix("uniform", m, k, m, 1)
    B = synth.matrix("uniform", k, n, k, 2)
    a = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, 6, kseg=8192)
    b = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, 6, kseg=64)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m)
    assert first_mismatch(a, b, 16 * U * G, m) is None
    Ai = synth.matrix("int8", m, k, m, 3)
    Bi = synth.matrix("int8", k, n, k, 4)
    a = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, Ai, m, Bi, k, 0.0, None, m, 3, kseg=8192)
    b = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, Ai, m, Bi, k, 0.0, None, m, 3, kseg=7)
    assert np.array_equal(a, b)


def test_nonfinite_rows_and_columns(oracle_mod):
    m, n, k = 4, 3, 5
    A = synth.matrix("uniform", m, k, m, 1)
    B = synth.matrix("uniform", k, n, k, 2)
    A[2 * m + 1] = np.inf   # row 1 of A
    B[2 * k + 4] = np.nan   # column 2 of B
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, 4).reshape(n, m).T
    assert np.isnan(out[1, :]).all() and np.isnan(out[:, 2]).all()
    assert np.isfinite(np.delete(np.delete(out, 1, axis=0), 2, axis=1)).all()


def test_quick_returns_and_codes(oracle_mod):
    m, n, k = 3, 2, 4
    C0 = synth.uniform_pm1(9, m * n)
    nan = np.full(64, np.nan)
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 0.0, nan, m, nan, k, 3.0, C0, m, 4)
    assert np.array_equal(out, 3.0 * C0)
    with pytest.raises(ValueError):
        oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, nan, m, nan, k, 0.0, None, m, 10)
    with pytest.raises(ValueError):
        oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, nan, 2, nan, k, 0.0, None, m, 4)


def test_one_level_group_rounds_once(oracle_mod):
    # 14-bit integers with every row/column maximum in [2^13, 2^14) split into exactly two
    # 7-bit digits, so with three slices no non-zero digit product is dropped and levels
    # 2..4 form one group.  With one segment the whole product is then summed exactly and
    # rounded once onto beta*C0 (itself rounded first): the result is
    # alpha*A*B + fl(beta*C0) correctly rounded.  beta*C0 is of
    # the size of the result, so rounding after each level (or a wrong scale for the
    # group) moves some entries by an ulp.
    m, n, k = 7, 6, 300
    Ai = synth.small_ints(11, m * k, -(2 ** 14 - 1), 2 ** 14 - 1).reshape(k, m).T.copy()
    Bi = synth.small_ints(12, k * n, -(2 ** 14 - 1), 2 ** 14 - 1).reshape(n, k).T.copy()
    Ai[:, 0] = 2.0 ** 13 + 5   # row maxima (exponent 14)
    Bi[0, :] = -(2.0 ** 13 + 3)  # column maxima
    C0 = synth.matrix("uniform", m, n, m, 13) * 2.0 ** 37
    alpha, beta = 0.7, -0.3
    A = Ai.flatten(order="F")
    B = Bi.flatten(order="F")
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, alpha, A, m, B, k, beta, C0, m, 3)
    S = Ai.astype(np.int64) @ Bi.astype(np.int64)
    for i in range(m):
        for j in range(n):
            want = float(Fraction(alpha) * int(S[i, j]) + Fraction(beta * float(C0[j * m + i])))
            assert out[j * m + i] == want, (i, j)


def test_scale_split_keeps_results_near_underflow_exact(oracle_mod):
    # Integers up to 8 in magnitude scaled by 2^-510: one 7-bit digit holds them exactly, and the
    # result alpha x (integer product) x 2^-1020 is a normal number, so the method gives it
    # correctly rounded.  alpha 2^(sigma_i + tau_j - 14) = 0.7 x 2^-1026 would be subnormal and
    # lose bits of alpha, so the power of two has to be split between alpha 2^(tau_j - 14) and
    # P 2^sigma_i.
    m, n, k = 9, 7, 200
    alpha = 0.7
    A = synth.matrix("int8", m, k, m, 31) * 2.0 ** -510
    B = synth.matrix("int8", k, n, k, 32) * 2.0 ** -510
    Ai = np.rint(synth.view(A, m, k, m) * 2.0 ** 510).astype(np.int64)
    Bi = np.rint(synth.view(B, k, n, k) * 2.0 ** 510).astype(np.int64)
    S = Ai @ Bi
    assert np.abs(S).max() < 2 ** 53 and np.all(np.abs(S[S != 0]) >= 2)
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, alpha, A, m, B, k, 0.0, None, m, 1)
    for i in range(m):
        for j in range(n):
            want = float(Fraction(alpha) * int(S[i, j]) * Fraction(1, 2 ** 1020))
            assert out[j * m + i] == want, (i, j)
