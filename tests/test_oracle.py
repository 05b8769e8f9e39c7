"""Pins of the plain CPU oracle (oracle/oracle.c) against things other than itself:
the paper's worked example, closed forms, exact integer and rational arithmetic,
an independent library product, and the quick-return rules of the BLAS.

The operation is the dgemm of the paper, Section 1.2; storage is column-major
with leading dimensions, Section 2.1.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

from conftest import U, first_mismatch, frac_dot_rows
from paper_1609_00076_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _read_golden(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = rest
    return vals


def _stored(ta, rows, cols):
    """(stored rows, stored cols) of op(X) = rows x cols."""
    return (cols, rows) if ta else (rows, cols)


def _rand(kind, rows, cols, seed, pad=0, e=0):
    ld = rows + pad
    return synth.matrix(kind, rows, cols, ld, seed, e=e), ld


# --------------------------------------------------------------------------
# the paper's worked example (Section 1.2): interior pointer, lda = 3
# --------------------------------------------------------------------------
def test_leading_dimension_example(oracle_mod):
    g = _read_golden("ld_example.txt")
    arr = np.array([float(x) for x in g["array"]])
    off, lda = int(g["offset"][0]), int(g["lda"][0])
    rows, cols = int(g["rows"][0]), int(g["cols"][0])
    sub = np.array([float(x) for x in g["submatrix"]]).reshape(rows, cols)
    A = arr[off:].copy()  # the interior pointer: A points at 1.2
    # op(A) * I == the sub-matrix, bit for bit
    eye = np.array([1.0, 0.0, 0.0, 1.0])
    C = np.full(4, np.nan)
    out = oracle_mod.dgemm_rows("N", "N", rows, cols, rows, 1.0, A, lda, eye, 2, 0.0, C, 2)
    assert np.array_equal(out.reshape(cols, rows).T, sub)
    # op(A)^T * I == the transposed sub-matrix
    out = oracle_mod.dgemm_rows("T", "N", rows, cols, rows, 1.0, A, lda, eye, 2, 0.0, C, 2)
    assert np.array_equal(out.reshape(cols, rows).T, sub.T)
    # op(A) * op(A) against exact rational arithmetic on the stored doubles
    out = oracle_mod.dgemm_rows("N", "N", rows, cols, rows, 1.0, A, lda, A, lda, 0.0, C, 2)
    exact = frac_dot_rows(False, False, rows, cols, rows, 1.0, A, lda, A, lda, 0.0, C, 2)
    for i in range(rows):
        for j in range(cols):
            assert out[j * rows + i] == float(exact[i][j])  # correctly rounded
    # and with the values written out by hand: 1.2*1.2 + 1.3*2.2, ...
    assert abs(out[0] - (1.2 * 1.2 + 1.3 * 2.2)) <= 4 * U * 4.3


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 3), (33, 17, 129)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (1.5, -0.5), (-3.25, 2.0)])
def test_all_ones(oracle_mod, m, n, k, alpha, beta):
    A = np.ones(m * k)
    B = np.ones(k * n)
    C0 = synth.uniform_pm1(11, m * n)
    out = oracle_mod.dgemm_rows("N", "N", m, n, k, alpha, A, m, B, k, beta, C0, m)
    for idx in range(m * n):
        exact = Fraction(alpha) * k + (Fraction(beta) * Fraction(float(C0[idx])) if beta else 0)
        assert out[idx] == float(exact), idx


@pytest.mark.parametrize("ta", ["N", "T"])
@pytest.mark.parametrize("tb", ["N", "T"])
def test_identity(oracle_mod, ta, tb):
    m = k = 9
    n = 6
    alpha, beta = 1.5, -0.75
    I = np.eye(k).flatten(order="F")
    rb, cb = _stored(tb == "T", k, n)
    B, ldb = _rand("uniform", rb, cb, 5, pad=2)
    C0 = synth.uniform_pm1(6, m * n)
    out = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, I, k, B, ldb, beta, C0, m)
    Bop = synth.view(B, rb, cb, ldb)
    Bop = Bop.T if tb == "T" else Bop
    for i in range(m):
        for j in range(n):
            exact = Fraction(alpha) * Fraction(float(Bop[i, j])) + Fraction(beta) * Fraction(float(C0[j * m + i]))
            assert abs(Fraction(out[j * m + i]) - exact) <= Fraction(U) * abs(exact)


def test_permutation(oracle_mod):
    m = k = 13
    n = 8
    perm = np.array([(5 * i + 3) % m for i in range(m)])
    P = np.zeros((m, k))
    P[np.arange(m), perm] = 1.0
    B, ldb = _rand("uniform", k, n, 21, pad=3)
    out = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, P.flatten(order="F"), m, B, ldb, 0.0, None, m)
    expect = synth.view(B, k, n, ldb)[perm, :]
    assert np.array_equal(out.reshape(n, m).T, expect)
    # the same permutation from the right permutes columns
    Q = np.zeros((n, n))
    qp = np.array([(3 * j + 1) % n for j in range(n)])
    Q[qp, np.arange(n)] = 1.0
    A, lda = _rand("uniform", m, n, 22)
    out = oracle_mod.dgemm_rows("N", "N", m, n, n, 1.0, A, lda, Q.flatten(order="F"), n, 0.0, None, m)
    assert np.array_equal(out.reshape(n, m).T, synth.view(A, m, n, lda)[:, qp])


# --------------------------------------------------------------------------
# transposes: against explicit transposition and an independent library product
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ta", ["N", "T", "t", "C"])
@pytest.mark.parametrize("tb", ["N", "n", "T", "c"])
def test_transposes(oracle_mod, ta, tb):
    m, n, k = 23, 19, 31
    alpha, beta = 1.5, -0.5
    ra, ca = _stored(ta in "TtCc", m, k)
    rb, cb = _stored(tb in "TtCc", k, n)
    A, lda = _rand("uniform", ra, ca, 31, pad=4)
    B, ldb = _rand("uniform", rb, cb, 32, pad=2)
    C0, ldc = _rand("uniform", m, n, 33, pad=1)
    out = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    Aop = synth.view(A, ra, ca, lda)
    Aop = Aop.T if ta in "TtCc" else Aop
    Bop = synth.view(B, rb, cb, ldb)
    Bop = Bop.T if tb in "TtCc" else Bop
    # explicit transposition -> the 'N','N' call sees the same numbers in the same order
    An = np.ascontiguousarray(Aop.T).flatten()  # column-major m x k, ld = m
    Bn = np.ascontiguousarray(Bop.T).flatten()
    ref = oracle_mod.dgemm_rows("N", "N", m, n, k, alpha, An, m, Bn, k, beta, C0, ldc)
    assert first_mismatch(out, ref, None, m) is None
    # numpy's product, an independent implementation, within the FP64 bound
    npref = (alpha * (Aop @ Bop) + beta * synth.view(C0, m, n, ldc)).flatten(order="F")
    G = (abs(alpha) * (np.abs(Aop) @ np.abs(Bop)) + abs(beta) * np.abs(synth.view(C0, m, n, ldc))).flatten(order="F")
    assert first_mismatch(out, npref, 2 * (k + 2) * U * G, m) is None
    # exact rational arithmetic on a corner
    exact = frac_dot_rows(ta in "TtCc", tb in "TtCc", 3, 3, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    for i in range(3):
        for j in range(3):
            assert abs(Fraction(out[j * m + i]) - exact[i][j]) <= Fraction(2 * U) * abs(exact[i][j])


def test_integer_inputs_exact(oracle_mod):
    m, n, k = 40, 36, 300
    A, lda = _rand("int8", m, k, 41)
    B, ldb = _rand("int8", k, n, 42)
    C0, ldc = _rand("int8", m, n, 43)
    Ai = synth.view(A, m, k, lda).astype(np.int64)
    Bi = synth.view(B, k, n, ldb).astype(np.int64)
    Ci = synth.view(C0, m, n, ldc).astype(np.int64)
    out = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C0, ldc)
    assert np.array_equal(out.reshape(n, m).T, (Ai @ Bi).astype(np.float64))
    out = oracle_mod.dgemm_rows("N", "N", m, n, k, 2.0, A, lda, B, ldb, -3.0, C0, ldc)
    assert np.array_equal(out.reshape(n, m).T, (2 * (Ai @ Bi) - 3 * Ci).astype(np.float64))


# --------------------------------------------------------------------------
# the compensated accumulation
# --------------------------------------------------------------------------
def test_dot2_cancellation(oracle_mod):
    # naive summation returns 0 here; the exact value is 1 + 2^-30
    x = np.array([2.0 ** 60, 1.0, -(2.0 ** 60), 2.0 ** -30])
    y = np.ones(4)
    out = oracle_mod.dgemm_rows("N", "N", 1, 1, 4, 1.0, x, 1, y, 4, 0.0, None, 1)
    assert out[0] == 1.0 + 2.0 ** -30


def test_dot2_ill_conditioned_vs_rational(oracle_mod):
    rng_vals = synth.uniform_pm1(77, 400)
    k = 100
    # pairs (v, -v) scaled large plus small remainders: condition number ~ 1e25
    a = np.empty(k)
    b = np.empty(k)
    for p in range(0, k, 2):
        big = np.ldexp(rng_vals[p], 40 + (p % 17))
        a[p], b[p] = big, 1.0 + rng_vals[p + 1] * 2.0 ** -20
        a[p + 1], b[p + 1] = -big, 1.0 + rng_vals[p + 1] * 2.0 ** -20 + 2.0 ** -52
    out = oracle_mod.dgemm_rows("T", "N", 1, 1, k, 1.0, a, k, b, k, 0.0, None, 1)
    exact = sum((Fraction(float(a[p])) * Fraction(float(b[p])) for p in range(k)), Fraction(0))
    absum = sum((abs(Fraction(float(a[p])) * Fraction(float(b[p]))) for p in range(k)), Fraction(0))
    naive = float(np.dot(a, b))
    # Dot2 bound (Ogita-Rump-Oishi 2005, Prop. 5.5): u|s| + gamma_k^2 sum|a b|
    gam = k * U / (1 - k * U)
    bound = Fraction(U) * abs(exact) + Fraction(gam * gam) * absum
    assert abs(Fraction(out[0]) - exact) <= bound
    assert abs(Fraction(naive) - exact) > bound  # the naive sum would fail this pin


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_rational(oracle_mod, seed):
    z = synth.splitmix64(900 + seed, 8)
    m, n, k = 1 + int(z[0] % 4), 1 + int(z[1] % 4), 1 + int(z[2] % 6)
    ta, tb = ("N", "T")[int(z[3] % 2)], ("N", "T")[int(z[4] % 2)]
    alpha = float(synth.uniform_pm1(seed, 1)[0] * 3)
    beta = float(synth.uniform_pm1(seed + 50, 1)[0] * 2)
    ra, ca = _stored(ta == "T", m, k)
    rb, cb = _stored(tb == "T", k, n)
    A, lda = _rand("scaled", ra, ca, seed + 1, pad=1, e=20)
    B, ldb = _rand("scaled", rb, cb, seed + 2, pad=0, e=20)
    C0, ldc = _rand("uniform", m, n, seed + 3, pad=2)
    out = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    exact = frac_dot_rows(ta == "T", tb == "T", m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    for i in range(m):
        for j in range(n):
            err = abs(Fraction(out[j * m + i]) - exact[i][j])
            assert err <= Fraction(2 * U) * abs(exact[i][j]) + Fraction(4 * (k * U) ** 2) * Fraction(G[j * m + i])


# --------------------------------------------------------------------------
# quick returns and argument checks (reference-BLAS conventions)
# --------------------------------------------------------------------------
def test_quick_returns(oracle_mod):
    m, n, k = 5, 4, 3
    Anan = np.full(m * k, np.nan)
    Bnan = np.full(k * n, np.nan)
    C0 = synth.uniform_pm1(3, m * n)
    # alpha == 0: A and B are not read, C := beta*C
    out = oracle_mod.dgemm_rows("N", "N", m, n, k, 0.0, Anan, m, Bnan, k, -2.0, C0, m)
    assert np.array_equal(out, -2.0 * C0)
    # k == 0: C := beta*C
    out = oracle_mod.dgemm_rows("N", "N", m, n, 0, 1.0, Anan, m, Bnan, 1, 0.5, C0, m)
    assert np.array_equal(out, 0.5 * C0)
    # beta == 0: C is not read, NaN in C does not propagate
    A = synth.uniform_pm1(4, m * k)
    B = synth.uniform_pm1(5, k * n)
    out = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, np.full(m * n, np.nan), m)
    assert np.isfinite(out).all()
    # alpha == 0 and beta == 0: zeros without reading anything
    out = oracle_mod.dgemm_rows("N", "N", m, n, k, 0.0, Anan, m, Bnan, k, 0.0, np.full(m * n, np.nan), m)
    assert np.array_equal(out, np.zeros(m * n))
    # in-place form: m == 0 leaves C untouched
    C = C0.copy()
    assert oracle_mod.dgemm("N", "N", 0, n, k, 1.0, A, 1, B, k, 0.0, C, 1) == 0
    assert np.array_equal(C, C0)


@pytest.mark.parametrize("args,code", [
    (("X", "N", 2, 2, 2, 2, 2, 2), 1), (("N", "Q", 2, 2, 2, 2, 2, 2), 2),
    (("N", "N", -1, 2, 2, 2, 2, 2), 3), (("N", "N", 2, -1, 2, 2, 2, 2), 4),
    (("N", "N", 2, 2, -1, 2, 2, 2), 5), (("N", "N", 3, 2, 2, 2, 2, 3), 8),
    (("T", "N", 2, 2, 3, 2, 3, 2), 8), (("N", "N", 2, 2, 3, 2, 2, 2), 10),
    (("N", "T", 2, 3, 2, 2, 2, 2), 10), (("N", "N", 3, 2, 2, 3, 2, 2), 13),
])
def test_argument_codes(oracle_mod, args, code):
    ta, tb, m, n, k, lda, ldb, ldc = args
    buf = np.zeros(64)
    C = np.zeros(64)
    assert oracle_mod.dgemm(ta, tb, m, n, k, 1.0, buf, lda, buf, ldb, 0.0, C, ldc) == code


def test_rows_subset_matches_full(oracle_mod):
    m, n, k = 30, 11, 17
    A, lda = _rand("uniform", m, k, 61, pad=3)
    B, ldb = _rand("uniform", k, n, 62)
    C0, ldc = _rand("uniform", m, n, 63, pad=2)
    full = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C0, ldc)
    rows = [29, 0, 7, 7, 15]
    sub = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C0, ldc, rows=rows)
    assert np.array_equal(sub.reshape(n, len(rows)).T, full.reshape(n, m).T[rows, :])


def test_abs_bound(oracle_mod):
    m, n, k = 6, 5, 7
    A, lda = _rand("uniform", m, k, 71)
    B, ldb = _rand("uniform", k, n, 72)
    C0, ldc = _rand("uniform", m, n, 73)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, -1.5, A, lda, B, ldb, 0.25, C0, ldc)
    ref = 1.5 * np.abs(synth.view(A, m, k, lda)) @ np.abs(synth.view(B, k, n, ldb)) + 0.25 * np.abs(
        synth.view(C0, m, n, ldc))
    assert np.allclose(G.reshape(n, m).T, ref, rtol=4 * k * U, atol=0)
