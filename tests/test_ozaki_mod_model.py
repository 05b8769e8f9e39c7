"""Pins of the CPU model of the modular emulation (oracle/ozaki_mod_model.c).

The model restates Ozaki scheme II (Ozaki, Uchino and Imamura, 2025): rounded scaled
integers A', B' and their exact product C', then one conversion and one fused update.
These tests tie it to exact arithmetic: Python's exact integer-to-float conversion,
integer inputs, a closed form, the tie rule of the rounding to integers, a rational
a-priori bound, and the plain Dot2 oracle.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import synth


def test_int128_conversion_is_correctly_rounded(oracle_mod):
    rng = np.random.default_rng(5)
    cases = [0, 1, -1, 2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 60 + 2 ** 7), 2 ** 60 + 2 ** 7 + 1, 2 ** 100 + 2 ** 47,
             2 ** 100 + 3 * 2 ** 47, 2 ** 126 - 1, -(2 ** 126 - 1)]
    for _ in range(2000):
        bits = int(rng.integers(1, 127))
        v = int(rng.integers(0, 2 ** 62)) << max(0, bits - 62)
        v = v ^ int(rng.integers(0, 2 ** 31))
        cases.append(-v if rng.integers(0, 2) else v)
    for v in cases:
        assert oracle_mod.ozmod_i128_to_double(v) == float(v), v  # Python's float(int) rounds correctly


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_integer_inputs_exact(oracle_mod, ta, tb):
    m, n, k = 19, 17, 301
    ra, ca = (k, m) if ta == "T" else (m, k)
    rb, cb = (n, k) if tb == "T" else (k, n)
    A = synth.matrix("int8", ra, ca, ra + 2, 11)
    B = synth.matrix("int8", rb, cb, rb, 12)
    C0 = synth.matrix("int8", m, n, m + 1, 13)
    Ai = synth.view(A, ra, ca, ra + 2).astype(np.int64)
    Bi = synth.view(B, rb, cb, rb).astype(np.int64)
    Ai = Ai.T if ta == "T" else Ai
    Bi = Bi.T if tb == "T" else Bi
    Ci = synth.view(C0, m, n, m + 1).astype(np.int64)
    out = oracle_mod.ozmod_dgemm_rows(ta, tb, m, n, k, 2.0, A, ra + 2, B, rb, -1.0, C0, m + 1, 20)
    assert np.array_equal(out.reshape(n, m).T, (2 * (Ai @ Bi) - Ci).astype(np.float64))


def test_all_ones_closed_form(oracle_mod):
    m, n, k = 5, 6, 1000
    out = oracle_mod.ozmod_dgemm_rows("N", "N", m, n, k, 1.5, np.ones(m * k), m, np.ones(k * n), k, 0.0, None, m,
                                      30)
    assert np.all(out == 1.5 * k)


def test_rounding_to_integers_is_ties_to_even(oracle_mod):
    # a = 0.5 + 2^-(t+1): sigma = 0, a 2^t = 2^(t-1) + 1/2, a tie.  Ties to even give
    # A' = 2^(t-1) and the result 0.5 exactly; rounding half up would give 0.5 + 2^-t.
    t = 10
    a = 0.5 + 2.0 ** -(t + 1)
    out = oracle_mod.ozmod_dgemm_rows("N", "N", 1, 1, 1, 1.0, np.array([a]), 1, np.array([1.0]), 1, 0.0, None, 1, t)
    assert out[0] == 0.5
    # a = 0.5 + 3 * 2^-(t+1): a 2^t = 2^(t-1) + 3/2 rounds to the even 2^(t-1) + 2
    a = 0.5 + 3 * 2.0 ** -(t + 1)
    out = oracle_mod.ozmod_dgemm_rows("N", "N", 1, 1, 1, 1.0, np.array([a]), 1, np.array([1.0]), 1, 0.0, None, 1, t)
    assert out[0] == 0.5 + 2.0 ** -(t - 1)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("t", [8, 13, 21])
def test_error_bound_vs_rationals(oracle_mod, seed, t):
    m, n, k = 4, 3, 11
    A = synth.matrix("scaled", m, k, m, 400 + seed, e=10)
    B = synth.matrix("scaled", k, n, k, 500 + seed, e=10)
    alpha = 1.25
    out = oracle_mod.ozmod_dgemm_rows("N", "N", m, n, k, alpha, A, m, B, k, 0.0, None, m, t)

    def a(i, p):
        return float(A[p * m + i])

    def b(p, j):
        return float(B[j * k + p])

    sig = [max(oracle_mod.ozaki_exponent(a(i, p)) for p in range(k) if a(i, p) != 0) for i in range(m)]
    tau = [max(oracle_mod.ozaki_exponent(b(p, j)) for p in range(k) if b(p, j) != 0) for j in range(n)]
    for i in range(m):
        mu = sum(abs(Fraction(a(i, p))) for p in range(k)) / Fraction(2) ** sig[i]
        for j in range(n):
            nu = sum(abs(Fraction(b(p, j))) for p in range(k)) / Fraction(2) ** tau[j]
            exact = Fraction(alpha) * sum(Fraction(a(i, p)) * Fraction(b(p, j)) for p in range(k))
            bound = abs(Fraction(alpha)) * Fraction(2) ** (sig[i] + tau[j] - t - 1) * (
                mu + nu + k * Fraction(1, 2 ** (t + 1)))
            tol = bound + 3 * Fraction(U) * (abs(exact) + bound)  # plus the conversion and the fma
            assert abs(Fraction(out[j * m + i]) - exact) <= tol, (i, j)


@pytest.mark.parametrize("e", [0, 8])
def test_fp64_bound_at_44_bits(oracle_mod, e):
    m, n, k = 40, 36, 384
    A = synth.matrix("scaled", m, k, m + 1, 600 + e, e=e)
    B = synth.matrix("scaled", k, n, k, 700 + e, e=e)
    C0 = synth.matrix("uniform", m, n, m, 800 + e)
    ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.5, A, m + 1, B, k, -0.5, C0, m)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.5, A, m + 1, B, k, -0.5, C0, m)
    out = oracle_mod.ozmod_dgemm_rows("N", "N", m, n, k, 1.5, A, m + 1, B, k, -0.5, C0, m, 48)
    assert first_mismatch(out, ref, 2 * k * U * G, m) is None


def test_quick_returns_and_codes(oracle_mod):
    z = np.zeros(16)
    with pytest.raises(ValueError, match="status 1"):
        oracle_mod.ozmod_dgemm_rows("X", "N", 2, 2, 2, 1.0, z, 2, z, 2, 0.0, z, 2, 20)
    with pytest.raises(ValueError, match="status 18"):
        oracle_mod.ozmod_dgemm_rows("N", "N", 2, 2, 2, 1.0, z, 2, z, 2, 0.0, z, 2, 63)
    C0 = np.arange(4.0)
    out = oracle_mod.ozmod_dgemm_rows("N", "N", 2, 2, 0, 1.0, z, 2, z, 1, 3.0, C0, 2, 20)
    assert np.array_equal(out, 3.0 * C0)
