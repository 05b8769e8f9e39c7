"""GPU parity of the GEMM-based level-3 BLAS (gbd_dsyrk, gbd_dtrmm, gbd_dtrsm) with the oracle.

Three product paths (native FP64; emulated mode forced to the split emulation; emulated mode
forced to the modular emulation) run every side/uplo/trans/diag case at sizes that recurse
at least once.  Unreferenced triangles and unit diagonals hold NaN,
so reading them would show.  Tolerances:
  DSYRK  each element is one GEMM element: 2 k u G, G = |alpha||op(A)||op(A)^T| + |beta||C0|
         (the benchmark spec's bound of the product);
  DTRMM  an element is the sum of the products along the recursion, each within its own
         bound, plus one rounding per level: (2 order + 16) u G, G = |alpha||op(T)||B0|;
  DTRSM  the residual |op(T) X - alpha B0| <= 4 order u (|op(T)||X| + |alpha||B0|) (the
         substitution's backward error, times the recursion's levels), and the forward
         error against the oracle's solution on well-conditioned triangles.
"""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from conftest import U, DeviceBuf
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu
MODES = {"native": gbdgemm.GBD_MODE_NATIVE, "emulated": gbdgemm.GBD_MODE_EMULATED,
         "modular": gbdgemm.GBD_MODE_EMULATED}


@pytest.fixture
def products(monkeypatch):
    """Forces the product path of emulated mode at these small sizes: "emulated" sends every
    product to the split emulation, "modular" to the modular one (split where 16 moduli
    cannot reach the target)."""
    def force(mode):
        if mode == "emulated":
            monkeypatch.setenv("GBD_L3_NATIVE_FLOPS", "0")
            monkeypatch.setenv("GBD_L3_MODULAR_OUTPUTS", "1e300")
        elif mode == "modular":
            monkeypatch.setenv("GBD_L3_NATIVE_FLOPS", "0")
            monkeypatch.setenv("GBD_L3_MODULAR_OUTPUTS", "0")
    return force


def _ws(nbytes):
    import torch
    return torch.full((max(nbytes, 8) // 8 + 32,), float("nan"), dtype=torch.float64, device="cuda")


def _sync_ok():
    import torch
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0, gbdgemm.gbd_last_error()


def _tri(order, uplo, diag, seed, kind="uniform"):
    """Stored triangular A (ld = order + 3) with NaN outside its triangle (and on a unit
    diagonal), and the dense triangle it stands for.  Well conditioned: |diag| in [1, 2],
    off-diagonal entries uniform[-1, 1) / order."""
    lda = order + 3
    vals = synth.view(synth.matrix(kind, order, order, order, seed), order, order, order).copy()
    rng_d = synth.view(synth.matrix("uniform", order, 1, order, seed + 7), order, 1, order)[:, 0]
    if kind == "uniform":
        vals = vals / order
        np.fill_diagonal(vals, np.sign(rng_d + 1e-300) * (1.0 + np.abs(rng_d)))
    low = np.tril(np.ones((order, order), bool), -1)
    keep = low if uplo == "L" else low.T
    tri = np.where(keep, vals, 0.0)
    if diag == "U":
        np.fill_diagonal(tri, 1.0)
    else:
        np.fill_diagonal(tri, np.diag(vals))
    stored = np.where(keep, vals, np.nan)
    if diag == "N":
        np.fill_diagonal(stored, np.diag(vals))
    buf = np.full(lda * order, np.nan)
    for j in range(order):
        buf[j * lda: j * lda + order] = stored[:, j]
    return buf, lda, tri


# ---------------------------------------------------------------------------------- DSYRK
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_syrk_within_bound(oracle_mod, products, mode, uplo, trans):
    products(mode)
    n, k = 700, 300
    ra, ca = (n, k) if trans == "N" else (k, n)
    lda, ldc = ra + 2, n + 1
    A = synth.matrix("uniform", ra, ca, lda, 11)
    C0 = synth.matrix("uniform", n, n, ldc, 12)
    other = ~np.tril(np.ones((n, n), bool)) if uplo == "L" else ~np.triu(np.ones((n, n), bool))
    C0v = synth.view(C0, n, n, ldc)
    C0v[other] = np.nan  # the other triangle: never read for the result, never written
    ref = C0.copy()
    assert oracle_mod.dsyrk(uplo, trans, n, k, 1.5, A, lda, -0.5, ref, ldc) == 0
    dA, dC = DeviceBuf(A), DeviceBuf(C0)
    wsb = gbdgemm.gbd_dsyrk_workspace_size(n, k, MODES[mode])
    ws = _ws(wsb)
    rc = gbdgemm.gbd_dsyrk(uplo, trans, n, k, 1.5, dA.ptr, lda, -0.5, dC.ptr, ldc, MODES[mode], 0.0, ws, wsb)
    assert rc == 0, gbdgemm.gbd_last_error()
    _sync_ok()
    assert dA.guards_intact() and dC.guards_intact()
    got = synth.view(dC.host(), n, n, ldc)
    op = synth.view(A, ra, ca, lda)
    op = op if trans == "N" else op.T
    G = 1.5 * np.abs(op) @ np.abs(op).T + 0.5 * np.abs(np.nan_to_num(C0v))
    tri = ~other
    assert np.all(np.isnan(got[other]))
    err = np.abs(got[tri] - synth.view(ref, n, n, ldc)[tri])
    assert np.all(err <= 2 * k * U * G[tri]), float(np.max(err / (2 * k * U * G[tri])))


@pytest.mark.parametrize("kernel,n", [("single", 700), ("pair", 700), ("pair", 3022)])
@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_syrk_modular_triangle(oracle_mod, products, monkeypatch, kernel, n, uplo, trans):
    # emulated DSYRK as one modular product over the tiles that meet the triangle, on the one-SM
    # and two-SM kernels; at n = 3022 the 78 tiles of 256 x 256 leave a last wave of 2 tiles,
    # which runs as one-SM quarters
    products("modular")
    monkeypatch.setenv("GBD_EMU_KERNEL", kernel)
    k = 300 if n < 1000 else 64
    ra, ca = (n, k) if trans == "N" else (k, n)
    lda, ldc = ra + 1, n + 3
    A = synth.matrix("uniform", ra, ca, lda, 15)
    C0 = synth.matrix("uniform", n, n, ldc, 16)
    other = ~np.tril(np.ones((n, n), bool)) if uplo == "L" else ~np.triu(np.ones((n, n), bool))
    C0v = synth.view(C0, n, n, ldc)
    C0v[other] = np.nan
    ref = C0.copy()
    assert oracle_mod.dsyrk(uplo, trans, n, k, -0.5, A, lda, 2.0, ref, ldc) == 0
    dA, dC = DeviceBuf(A), DeviceBuf(C0)
    wsb = gbdgemm.gbd_dsyrk_workspace_size(n, k, 1)
    assert wsb >= gbdgemm.gbd_dgemm_emu_mod_workspace_size(n, n, k, 0)
    ws = _ws(wsb)
    assert gbdgemm.gbd_dsyrk(uplo, trans, n, k, -0.5, dA.ptr, lda, 2.0, dC.ptr, ldc, 1, 0.0, ws, wsb) == 0
    _sync_ok()
    assert dA.guards_intact() and dC.guards_intact()
    got = synth.view(dC.host(), n, n, ldc)
    op = synth.view(A, ra, ca, lda)
    op = op if trans == "N" else op.T
    G = 0.5 * np.abs(op) @ np.abs(op).T + 2.0 * np.abs(np.nan_to_num(C0v))
    tri = ~other
    assert np.all(np.isnan(got[other]))
    err = np.abs(got[tri] - synth.view(ref, n, n, ldc)[tri])
    assert np.all(err <= 2 * k * U * G[tri]), float(np.max(err / (2 * k * U * G[tri])))


def test_syrk_large_emulated_within_bound(oracle_mod):
    # the 2048 x 2048 coupling block (4.2e6 outputs) goes to the modular emulation
    n, k = 4096, 256
    A = synth.matrix("uniform", n, k, n, 13)
    C0 = synth.matrix("uniform", n, n, n, 14)
    ref = C0.copy()
    assert oracle_mod.dsyrk("L", "N", n, k, 1.0, A, n, 1.0, ref, n) == 0
    dA, dC = DeviceBuf(A), DeviceBuf(C0)
    wsb = gbdgemm.gbd_dsyrk_workspace_size(n, k, 1)
    assert wsb >= gbdgemm.gbd_dgemm_emu_mod_workspace_size(2048, 2048, k, 0)
    ws = _ws(wsb)
    assert gbdgemm.gbd_dsyrk("L", "N", n, k, 1.0, dA.ptr, n, 1.0, dC.ptr, n, 1, 0.0, ws, wsb) == 0
    _sync_ok()
    got = synth.view(dC.host(), n, n, n)
    Av = synth.view(A, n, k, n)
    G = np.abs(Av) @ np.abs(Av).T + np.abs(synth.view(C0, n, n, n))
    low = np.tril(np.ones((n, n), bool))
    err = np.abs(got - synth.view(ref, n, n, n))[low]
    assert np.all(err <= 2 * k * U * G[low]), float(np.max(err / (2 * k * U * G[low])))


def test_syrk_integer_exact_native():
    n, k = 600, 257
    A = synth.matrix("int8", n, k, n, 21)
    C0 = synth.matrix("int8", n, n, n, 22)
    dA, dC = DeviceBuf(A), DeviceBuf(C0)
    wsb = gbdgemm.gbd_dsyrk_workspace_size(n, k, 0)
    ws = _ws(wsb)
    assert gbdgemm.gbd_dsyrk("L", "N", n, k, 2.0, dA.ptr, n, -1.0, dC.ptr, n, 0, 0.0, ws, wsb) == 0
    _sync_ok()
    Ai = synth.view(A, n, k, n).astype(np.int64)
    want = 2 * (Ai @ Ai.T) - synth.view(C0, n, n, n).astype(np.int64)
    got = synth.view(dC.host(), n, n, n)
    low = np.tril(np.ones((n, n), bool))
    assert np.array_equal(got[low], want[low].astype(np.float64))
    assert np.array_equal(got[~low], synth.view(C0, n, n, n)[~low])


# ---------------------------------------------------------------------------------- DTRMM
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("side,uplo,trans,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_trmm_within_bound(oracle_mod, products, mode, side, uplo, trans, diag):
    products(mode)
    order, other = 600, 150
    m, n = (order, other) if side == "L" else (other, order)
    A, lda, tri = _tri(order, uplo, diag, 31 + ord(side) + 2 * ord(uplo))
    ldb = m + 1
    B0 = synth.matrix("uniform", m, n, ldb, 32)
    ref = B0.copy()
    assert oracle_mod.dtrmm(side, uplo, trans, diag, m, n, -1.25, A, lda, ref, ldb) == 0
    dA, dB = DeviceBuf(A), DeviceBuf(B0)
    wsb = gbdgemm.gbd_dtrmm_workspace_size(side, m, n, MODES[mode])
    ws = _ws(wsb)
    rc = gbdgemm.gbd_dtrmm(side, uplo, trans, diag, m, n, -1.25, dA.ptr, lda, dB.ptr, ldb, MODES[mode], 0.0, ws, wsb)
    assert rc == 0, gbdgemm.gbd_last_error()
    _sync_ok()
    assert dA.guards_intact() and dB.guards_intact()
    got = synth.view(dB.host(), m, n, ldb)
    op = tri.T if trans == "T" else tri
    Bv = synth.view(B0, m, n, ldb)
    G = 1.25 * (np.abs(op) @ np.abs(Bv) if side == "L" else np.abs(Bv) @ np.abs(op))
    err = np.abs(got - synth.view(ref, m, n, ldb))
    tol = (2 * order + 16) * U * G
    assert np.all(err <= tol), float(np.max(err / tol))


# ---------------------------------------------------------------------------------- DTRSM
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("side,uplo,trans,diag", list(itertools.product("LR", "LU", "NT", "NU")))
def test_trsm_residual_and_forward(oracle_mod, products, mode, side, uplo, trans, diag):
    products(mode)
    order, other = 333, 130
    m, n = (order, other) if side == "L" else (other, order)
    A, lda, tri = _tri(order, uplo, diag, 41 + ord(side) + 2 * ord(trans))
    ldb = m + 2
    B0 = synth.matrix("uniform", m, n, ldb, 42)
    alpha = 0.75
    ref = B0.copy()
    assert oracle_mod.dtrsm(side, uplo, trans, diag, m, n, alpha, A, lda, ref, ldb) == 0
    dA, dB = DeviceBuf(A), DeviceBuf(B0)
    wsb = gbdgemm.gbd_dtrsm_workspace_size(side, m, n, MODES[mode])
    ws = _ws(wsb)
    rc = gbdgemm.gbd_dtrsm(side, uplo, trans, diag, m, n, alpha, dA.ptr, lda, dB.ptr, ldb, MODES[mode], 0.0, ws,
                           wsb)
    assert rc == 0, gbdgemm.gbd_last_error()
    _sync_ok()
    assert dA.guards_intact() and dB.guards_intact()
    X = dB.host()
    Xv = synth.view(X, m, n, ldb)
    # residual op(T) X - alpha B0, with op(T) X from the oracle's DTRMM (Dot2, one rounding)
    prod = X.copy()
    assert oracle_mod.dtrmm(side, uplo, trans, diag, m, n, 1.0, A, lda, prod, ldb) == 0
    Bv = synth.view(B0, m, n, ldb)
    R = np.abs(synth.view(prod, m, n, ldb) - alpha * Bv)
    op = tri.T if trans == "T" else tri
    G = (np.abs(op) @ np.abs(Xv) if side == "L" else np.abs(Xv) @ np.abs(op)) + abs(alpha) * np.abs(Bv)
    assert np.all(R <= 4 * order * U * G), float(np.max(R / (4 * order * U * G)))
    # forward error against the oracle's substitution (diagonally dominant, so well conditioned)
    Xr = synth.view(ref, m, n, ldb)
    scale = np.max(np.abs(Xr))
    assert np.max(np.abs(Xv - Xr)) <= 64 * order * U * scale


@pytest.mark.parametrize("side,trans", [("L", "N"), ("R", "T")])
def test_trsm_integer_exact_native(side, trans):
    # unit diagonal, small integers: every intermediate is an exact integer, so X is recovered
    order, other = 200, 96
    m, n = (order, other) if side == "L" else (other, order)
    A, lda, tri = _tri(order, "L", "U", 51, kind="int8")
    tri = np.rint(tri / 4).astype(np.int64)  # entries in [-2, 2]
    np.fill_diagonal(tri, 1)
    Ad = np.where(np.tril(np.ones((order, order), bool), -1), tri.astype(np.float64), np.nan)
    A = np.full(lda * order, np.nan)
    for j in range(order):
        A[j * lda: j * lda + order] = Ad[:, j]
    X = np.rint(synth.view(synth.matrix("int8", m, n, m, 52), m, n, m) / 2).astype(np.int64)
    op = tri.T if trans == "T" else tri
    Bd = (op @ X if side == "L" else X @ op)
    assert np.abs(Bd).max() < 2 ** 50
    B = synth.colmajor(m, n, m, Bd.astype(np.float64).flatten(order="F"), synth.SENTINEL)
    dA, dB = DeviceBuf(A), DeviceBuf(B)
    wsb = gbdgemm.gbd_dtrsm_workspace_size(side, m, n, 0)
    rc = gbdgemm.gbd_dtrsm(side, "L", trans, "U", m, n, 1.0, dA.ptr, lda, dB.ptr, m, 0, 0.0, None if wsb == 0 else
                           _ws(wsb), wsb)
    assert rc == 0, gbdgemm.gbd_last_error()
    _sync_ok()
    assert np.array_equal(synth.view(dB.host(), m, n, m), X.astype(np.float64))


def test_level3_quick_returns_and_errors():
    import torch
    nan = torch.full((4096,), float("nan"), dtype=torch.float64, device="cuda")
    B = torch.arange(64, dtype=torch.float64, device="cuda")
    # alpha = 0: B := 0 and A is not read
    assert gbdgemm.gbd_dtrsm("L", "L", "N", "N", 8, 8, 0.0, nan, 8, B, 8, 0, 0.0, None, 0) == 0
    assert gbdgemm.gbd_dtrmm("R", "U", "T", "U", 8, 8, 0.0, nan, 8, B, 8, 1, 0.0, None, 0) == 0
    _sync_ok()
    assert torch.count_nonzero(B).item() == 0
    # DSYRK with alpha = 0, beta = 0: the triangle becomes 0 without reading C
    C = torch.full((64,), float("nan"), dtype=torch.float64, device="cuda")
    assert gbdgemm.gbd_dsyrk("U", "N", 8, 4, 0.0, nan, 8, 0.0, C, 8, 0, 0.0, None, 0) == 0
    _sync_ok()
    Cm = C.cpu().numpy().reshape(8, 8).T
    assert np.all(Cm[np.triu(np.ones((8, 8), bool))] == 0.0) and np.all(np.isnan(Cm[~np.triu(np.ones((8, 8), bool))]))
    # a mode outside the two, and a missing workspace
    assert gbdgemm.gbd_dtrsm("L", "L", "N", "N", 8, 8, 1.0, nan, 8, B, 8, 7, 0.0, None, 0) == gbdgemm.GBD_ERR_ARG
    assert gbdgemm.gbd_dtrmm("L", "L", "N", "N", 8, 8, 1.0, nan, 8, B, 8, 0, 0.0, None, 0) == \
        gbdgemm.GBD_ERR_WORKSPACE
