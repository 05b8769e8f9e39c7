"""Pins of the level-3 oracle (oracle/level3.c): DSYRK, DTRMM, DTRSM by their definitions.

They are tied to exact arithmetic: integer inputs against numpy's int64 products (the
triangles built independently with np.tril/np.triu), closed forms, exact rational
solutions of tiny systems, the reference-BLAS quick returns and argument codes, and the
rule that the unreferenced triangle (and a unit diagonal) is never read (it holds NaN).
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np
import pytest

from conftest import U

SIDES, UPLOS, TRANS, DIAGS = "LR", "LU", "NT", "NU"


def _rng(seed):
    return np.random.default_rng(seed)


def _tri_stored(rng, order, uplo, diag, lo=-3, hi=4, dvals=(1.0, -1.0, 2.0, -2.0, 4.0)):
    """A triangular matrix A (order x order, column-major, ld = order + 1) holding NaN in its
    unreferenced triangle (and on a unit diagonal); returns (buffer, lda, dense triangle)."""
    lda = order + 1
    full = rng.integers(lo, hi, size=(order, order)).astype(np.float64)
    np.fill_diagonal(full, rng.choice(dvals, size=order))
    tri = np.tril(full) if uplo == "L" else np.triu(full)
    if diag == "U":
        np.fill_diagonal(tri, 1.0)
    stored = np.where(np.tril(np.ones((order, order))) if uplo == "L" else np.triu(np.ones((order, order))),
                      full, np.nan)
    if diag == "U":
        np.fill_diagonal(stored, np.nan)
    buf = np.full(lda * order, np.nan)
    for j in range(order):
        buf[j * lda: j * lda + order] = stored[:, j]
    return buf, lda, tri


def _mat(buf, rows, cols, ld):
    return np.array([buf[j * ld: j * ld + rows] for j in range(cols)]).T


def _buf(mat, ld, fill=np.nan):
    rows, cols = mat.shape
    out = np.full(ld * max(cols, 1), fill)
    for j in range(cols):
        out[j * ld: j * ld + rows] = mat[:, j]
    return out


# ---------------------------------------------------------------------------------- DSYRK
@pytest.mark.parametrize("uplo,trans", list(itertools.product(UPLOS, TRANS)))
def test_syrk_integer_exact_and_other_triangle_untouched(oracle_mod, uplo, trans):
    rng = _rng(1)
    n, k = 23, 17
    Ad = rng.integers(-8, 9, size=(n, k) if trans == "N" else (k, n)).astype(np.float64)
    lda = Ad.shape[0] + 2
    A = _buf(Ad, lda)
    C0 = rng.integers(-8, 9, size=(n, n)).astype(np.float64)
    C = _buf(C0, n + 1)
    assert oracle_mod.dsyrk(uplo, trans, n, k, 2.0, A, lda, -3.0, C, n + 1) == 0
    op = Ad if trans == "N" else Ad.T
    full = 2 * (op.astype(np.int64) @ op.T.astype(np.int64)) - 3 * C0.astype(np.int64)
    mask = np.tril(np.ones((n, n), bool)) if uplo == "L" else np.triu(np.ones((n, n), bool))
    got = _mat(C, n, n, n + 1)
    assert np.array_equal(got[mask], full[mask].astype(np.float64))
    assert np.array_equal(got[~mask], C0[~mask])


def test_syrk_all_ones_closed_form(oracle_mod):
    n, k = 9, 1000
    A = np.ones(n * k)
    C = np.full(n * n, 0.25)
    assert oracle_mod.dsyrk("L", "N", n, k, 1.5, A, n, 2.0, C, n) == 0
    got = _mat(C, n, n, n)
    assert np.all(got[np.tril(np.ones((n, n), bool))] == 1.5 * k + 0.5)


def test_syrk_rational_small(oracle_mod):
    rng = _rng(2)
    n, k = 4, 6
    Ad = rng.standard_normal((n, k))
    C0 = rng.standard_normal((n, n))
    C = _buf(C0, n)
    assert oracle_mod.dsyrk("U", "N", n, k, 0.7, _buf(Ad, n), n, -1.3, C, n) == 0
    got = _mat(C, n, n, n)
    for j in range(n):
        for i in range(j + 1):
            exact = Fraction(0.7) * sum(Fraction(Ad[i, p]) * Fraction(Ad[j, p]) for p in range(k)) + \
                Fraction(-1.3) * Fraction(C0[i, j])
            assert abs(Fraction(got[i, j]) - exact) <= 2 * Fraction(U) * abs(exact)


def test_syrk_quick_returns_and_codes(oracle_mod):
    n = 5
    A = np.full(n * n, np.nan)
    C = np.full(n * n, np.nan)
    assert oracle_mod.dsyrk("L", "N", n, 3, 0.0, A, n, 0.0, C, n) == 0  # beta = 0: C not read, A not read
    got = _mat(C, n, n, n)
    assert np.all(got[np.tril(np.ones((n, n), bool))] == 0.0)
    assert np.all(np.isnan(got[~np.tril(np.ones((n, n), bool))]))
    C2 = np.arange(n * n, dtype=np.float64)
    keep = C2.copy()
    assert oracle_mod.dsyrk("U", "T", n, 0, 1.0, A, 1, 1.0, C2, n) == 0
    assert np.array_equal(C2, keep)
    z = np.zeros(64)
    assert oracle_mod.dsyrk("X", "N", 2, 2, 1.0, z, 2, 0.0, z, 2) == 1
    assert oracle_mod.dsyrk("L", "X", 2, 2, 1.0, z, 2, 0.0, z, 2) == 2
    assert oracle_mod.dsyrk("L", "N", -1, 2, 1.0, z, 2, 0.0, z, 2) == 3
    assert oracle_mod.dsyrk("L", "N", 2, -1, 1.0, z, 2, 0.0, z, 2) == 4
    assert oracle_mod.dsyrk("L", "T", 2, 3, 1.0, z, 2, 0.0, z, 2) == 7
    assert oracle_mod.dsyrk("L", "N", 3, 2, 1.0, z, 3, 0.0, z, 2) == 10


# ---------------------------------------------------------------------------------- DTRMM
@pytest.mark.parametrize("side,uplo,trans,diag", list(itertools.product(SIDES, UPLOS, TRANS, DIAGS)))
def test_trmm_integer_exact(oracle_mod, side, uplo, trans, diag):
    rng = _rng(3)
    m, n = 19, 14
    order = m if side == "L" else n
    A, lda, tri = _tri_stored(rng, order, uplo, diag)
    Bd = rng.integers(-8, 9, size=(m, n)).astype(np.float64)
    B = _buf(Bd, m + 3)
    assert oracle_mod.dtrmm(side, uplo, trans, diag, m, n, 3.0, A, lda, B, m + 3) == 0
    op = (tri.T if trans == "T" else tri).astype(np.int64)
    want = 3 * (op @ Bd.astype(np.int64) if side == "L" else Bd.astype(np.int64) @ op)
    assert np.array_equal(_mat(B, m, n, m + 3), want.astype(np.float64))


def test_trmm_identity_and_zero_alpha(oracle_mod):
    m, n = 7, 5
    A = np.eye(m).flatten(order="F")
    Bd = _rng(4).standard_normal((m, n))
    B = _buf(Bd, m)
    assert oracle_mod.dtrmm("L", "U", "N", "N", m, n, 0.5, A, m, B, m) == 0
    assert np.array_equal(_mat(B, m, n, m), 0.5 * Bd)
    B = _buf(Bd, m)
    assert oracle_mod.dtrmm("R", "L", "T", "U", m, n, 0.0, np.full(n * n, np.nan), n, B, m) == 0
    assert np.all(_mat(B, m, n, m) == 0.0)


# ---------------------------------------------------------------------------------- DTRSM
@pytest.mark.parametrize("side,uplo,trans,diag", list(itertools.product(SIDES, UPLOS, TRANS, DIAGS)))
def test_trsm_recovers_integer_solutions_exactly(oracle_mod, side, uplo, trans, diag):
    # diagonals are +-1, +-2, +-4 (exact divisions), X integer, B = op(A) X or X op(A) exactly
    rng = _rng(5)
    m, n = 17, 12
    order = m if side == "L" else n
    A, lda, tri = _tri_stored(rng, order, uplo, diag, lo=-2, hi=3)
    X = rng.integers(-5, 6, size=(m, n)).astype(np.int64)
    op = (tri.T if trans == "T" else tri).astype(np.int64)
    Bd = (op @ X if side == "L" else X @ op).astype(np.float64)
    B = _buf(Bd, m + 1)
    assert oracle_mod.dtrsm(side, uplo, trans, diag, m, n, 1.0, A, lda, B, m + 1) == 0
    assert np.array_equal(_mat(B, m, n, m + 1), X.astype(np.float64))


@pytest.mark.parametrize("side,trans", [("L", "N"), ("R", "T")])
def test_trsm_rational_small(oracle_mod, side, trans):
    # a diagonally dominant 5 x 5 lower triangle: the exact rational solution, relative error <= 8 m u
    rng = _rng(6)
    order, other = 5, 3
    full = rng.standard_normal((order, order)) * 0.3
    np.fill_diagonal(full, 2.0 + rng.random(order))
    tri = np.tril(full)
    A = _buf(tri, order)
    m, n = (order, other) if side == "L" else (other, order)
    Bd = rng.standard_normal((m, n))
    B = _buf(Bd, m)
    alpha = 1.5
    assert oracle_mod.dtrsm(side, "L", trans, "N", m, n, alpha, A, order, B, m) == 0
    got = _mat(B, m, n, m)
    T = [[Fraction(tri[i, j]) for j in range(order)] for i in range(order)]
    op = [[T[j][i] for j in range(order)] for i in range(order)] if trans == "T" else T

    def solve_left(rhs):  # op x = rhs, exact, by elimination on the triangle op (lower or upper)
        low = all(op[i][j] == 0 for i in range(order) for j in range(i + 1, order))
        x = [Fraction(0)] * order
        seq = range(order) if low else range(order - 1, -1, -1)
        for i in seq:
            s = rhs[i] - sum(op[i][j] * x[j] for j in range(order) if j != i)
            x[i] = s / op[i][i]
        return x

    for u in range(other):
        if side == "L":
            exact = solve_left([Fraction(alpha) * Fraction(Bd[i, u]) for i in range(order)])
            vals = got[:, u]
        else:  # x op = alpha b  <=>  op^T x^T = alpha b^T
            opT = [[op[j][i] for j in range(order)] for i in range(order)]
            saved = op
            op = opT
            exact = solve_left([Fraction(alpha) * Fraction(Bd[u, i]) for i in range(order)])
            op = saved
            vals = got[u, :]
        for v, e in zip(vals, exact):
            assert abs(Fraction(v) - e) <= 8 * order * Fraction(U) * abs(e)


def test_trsm_unreferenced_parts_and_codes(oracle_mod):
    m, n = 6, 4
    A = np.full(m * m, np.nan)
    for j in range(m):
        for i in range(j + 1, m):
            A[j * m + i] = 0.5  # strictly lower part only; the diagonal (unit) and the upper part are NaN
    B = np.ones(m * n)
    assert oracle_mod.dtrsm("L", "L", "N", "U", m, n, 1.0, A, m, B, m) == 0
    assert np.all(np.isfinite(B))
    z = np.zeros(64)
    assert oracle_mod.dtrsm("X", "L", "N", "N", 2, 2, 1.0, z, 2, z, 2) == 1
    assert oracle_mod.dtrsm("L", "X", "N", "N", 2, 2, 1.0, z, 2, z, 2) == 2
    assert oracle_mod.dtrsm("L", "L", "X", "N", 2, 2, 1.0, z, 2, z, 2) == 3
    assert oracle_mod.dtrsm("L", "L", "N", "X", 2, 2, 1.0, z, 2, z, 2) == 4
    assert oracle_mod.dtrsm("L", "L", "N", "N", -1, 2, 1.0, z, 2, z, 2) == 5
    assert oracle_mod.dtrsm("L", "L", "N", "N", 2, -1, 1.0, z, 2, z, 2) == 6
    assert oracle_mod.dtrsm("R", "L", "N", "N", 2, 3, 1.0, z, 2, z, 2) == 9
    assert oracle_mod.dtrsm("L", "L", "N", "N", 3, 2, 1.0, z, 3, z, 2) == 11
    assert oracle_mod.dtrmm("L", "L", "N", "N", 3, 2, 1.0, z, 3, z, 2) == 11
