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


# --------------------------------------------------------------------------
# GPU helpers: run a library call on device copies of numpy buffers that are
# surrounded by guard bands of sentinel NaNs, and check the guards afterwards.
# --------------------------------------------------------------------------
GUARD = 64


class DeviceBuf:
    """A flat float64 device buffer holding `host` between two guard bands."""

    def __init__(self, host: np.ndarray | None, n: int | None = None, offset: int = 0):
        import torch
        from paper_1609_00076_gb300 import synth
        if host is None:
            host = np.full(n, synth.SENTINEL)
        self.n = host.size
        self.offset = offset  # extra elements between the guard and the data (alignment tests)
        full = np.full(GUARD + offset + self.n + GUARD, synth.SENTINEL)
        full[GUARD + offset: GUARD + offset + self.n] = host
        self.t = torch.from_numpy(full).cuda()

    @property
    def ptr(self) -> int:
        return self.t.data_ptr() + 8 * (GUARD + self.offset)

    def host(self) -> np.ndarray:
        full = self.t.cpu().numpy()
        return full[GUARD + self.offset: GUARD + self.offset + self.n].copy()

    def guards_intact(self) -> bool:
        from paper_1609_00076_gb300 import synth
        full = self.t.cpu().numpy().view(np.uint64)
        g1 = full[: GUARD + self.offset]
        g2 = full[GUARD + self.offset + self.n:]
        return bool((g1 == synth.SENTINEL_BITS).all() and (g2 == synth.SENTINEL_BITS).all())


def padding_intact(C: np.ndarray, m: int, n: int, ldc: int) -> bool:
    """Rows m..ldc-1 of every column still hold the sentinel (nothing wrote there)."""
    from paper_1609_00076_gb300 import synth
    if ldc == m or n == 0:
        return True
    v = C[: ldc * n].reshape(n, ldc)[:, m:].view(np.uint64)
    return bool((v == synth.SENTINEL_BITS).all())
