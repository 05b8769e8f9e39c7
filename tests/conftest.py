"""Shared fixtures and helpers of the test suite.

Markers: ``gpu`` marks every test that needs a GB300; everything else runs on a
CPU-only host (``pytest -m "not gpu"``).
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

U = 2.0 ** -53  # unit roundoff of FP64


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103, GB300)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def frac_dot_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc):
    """Exact rational alpha*op(A)*op(B) + beta*C0 (list of lists, m x n)."""
    def a(i, p):
        return Fraction(float(A[i * lda + p] if ta else A[p * lda + i]))

    def b(p, j):
        return Fraction(float(B[p * ldb + j] if tb else B[j * ldb + p]))

    out = []
    fa, fb = Fraction(float(alpha)), Fraction(float(beta))
    for i in range(m):
        row = []
        for j in range(n):
            s = sum((a(i, p) * b(p, j) for p in range(k)), Fraction(0))
            v = fa * s
            if beta != 0:
                v += fb * Fraction(float(C0[j * ldc + i]))
            row.append(v)
        out.append(row)
    return out


def first_mismatch(mine: np.ndarray, ref: np.ndarray, tol: np.ndarray | None, rows: int):
    """Report the first violating element in the style of a dgemm test driver:
    'C[i][j] != C_ref, mine, ref'.  Returns None when everything matches."""
    if tol is None:
        bad = ~((mine == ref) | (np.isnan(mine) & np.isnan(ref)))
    else:
        bad = ~(np.abs(mine - ref) <= tol)
    if not bad.any():
        return None
    idx = int(np.flatnonzero(bad)[0])
    i, j = idx % rows, idx // rows
    extra = "" if tol is None else f", tol {tol[idx]!r}"
    return f"C[{i}][{j}] != C_ref, {mine[idx]!r}, {ref[idx]!r}{extra} ({int(bad.sum())} bad)"
