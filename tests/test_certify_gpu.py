"""GPU tests of the certified precision choice of the emulations.

* The certification product (gbd_abs_product_lower_bound) is a lower bound of |op(A)||op(B)|
  element by element, close to it on well-scaled data, zero exactly where every term has a
  zero factor, and NaN in non-finite rows and columns.
* The automatic modes choose what the CPU statement of the rule (oracle/certify.c) chooses,
  or one step more (the device bounds |A||B| from below, the oracle evaluates it), and the
  results meet the componentwise FP64 bound of the Dot2 oracle.
* On the structured input whose magnitude sums misjudge |A||B| (half of every row of A and of
  every column of B scaled by 2^-30), the modular emulation refuses (bits = 0) or marks the
  call (bits = -1), and the split emulation and the grouped plans fall back to the FP64 path,
  whose result meets the bound.
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, DeviceBuf, first_mismatch
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def _stored(t, rows, cols):
    return (cols, rows) if t == "T" else (rows, cols)


def _inputs(kind, ta, tb, m, n, k, seed):
    ra, ca = _stored(ta, m, k)
    rb, cb = _stored(tb, k, n)
    if kind.startswith("halves"):
        d = int(kind[6:])
        A = synth.matrix("uniform", ra, ca, ra, seed)
        B = synth.matrix("uniform", rb, cb, rb, seed + 1)
        va, vb = A.reshape(ca, ra), B.reshape(cb, rb)
        if ta == "N":
            va[k // 2:, :] *= 2.0 ** -d
        else:
            va[:, k // 2:] *= 2.0 ** -d
        if tb == "N":
            vb[:, : k // 2] *= 2.0 ** -d
        else:
            vb[: k // 2, :] *= 2.0 ** -d
        return A, ra, B, rb
    if kind == "sparse":
        A = synth.matrix("uniform", ra, ca, ra, seed)
        B = synth.matrix("uniform", rb, cb, rb, seed + 1)
        A[synth.coin(seed + 2, A.size, 0.7)] = 0.0
        B[synth.coin(seed + 3, B.size, 0.7)] = 0.0
        return A, ra, B, rb
    if kind == "blocks":  # block-diagonal: whole blocks of |A||B| are exactly zero
        A = np.zeros(ra * ca)
        B = np.zeros(rb * cb)
        Am, Bm = synth.view(A, ra, ca, ra), synth.view(B, rb, cb, rb)
        opA = Am.T if ta == "T" else Am
        opB = Bm.T if tb == "T" else Bm
        opA[: m // 2, : k // 2] = synth.values("uniform", seed, (m // 2) * (k // 2)).reshape(m // 2, k // 2)
        opA[m // 2:, k // 2:] = synth.values("scaled", seed + 1, (m - m // 2) * (k - k // 2), 8).reshape(
            m - m // 2, k - k // 2)
        opB[: k // 2, : n // 2] = synth.values("uniform", seed + 2, (k // 2) * (n // 2)).reshape(k // 2, n // 2)
        opB[k // 2:, n // 2:] = synth.values("scaled", seed + 3, (k - k // 2) * (n - n // 2), 8).reshape(
            k - k // 2, n - n // 2)
        return A, ra, B, rb
    if kind == "extreme":  # magnitudes near both ends of the double range, in different rows
        A = synth.matrix("scaled", ra, ca, ra, seed, 8)
        B = synth.matrix("scaled", rb, cb, rb, seed + 1, 8)
        Am, Bm = synth.view(A, ra, ca, ra), synth.view(B, rb, cb, rb)
        opA = Am.T if ta == "T" else Am
        opB = Bm.T if tb == "T" else Bm
        opA[0, :] *= 2.0 ** -1000
        opA[1, :] *= 2.0 ** 900
        opB[:, 2] *= 2.0 ** -1030  # subnormal entries
        return A, ra, B, rb
    e = {"uniform": 0, "e8": 8, "e32": 32, "int8": 0}[kind]
    vk = "int8" if kind == "int8" else "scaled"
    return synth.matrix(vk, ra, ca, ra, seed, e), ra, synth.matrix(vk, rb, cb, rb, seed + 1, e), rb


def _lower_bound(ta, tb, m, n, k, A, lda, B, ldb, fp8=0):
    import torch
    dA, dB = DeviceBuf(A), DeviceBuf(B)
    dL = DeviceBuf(None, n=m * n)
    wsb = gbdgemm.gbd_abs_product_lower_bound_workspace_size(m, n, k)
    ws = torch.full((wsb // 8 + 64,), float("nan"), dtype=torch.float64, device="cuda")
    rc = gbdgemm.gbd_abs_product_lower_bound(ta, tb, m, n, k, dA.ptr, lda, dB.ptr, ldb, dL.ptr, m, fp8, ws, wsb)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    assert dA.guards_intact() and dB.guards_intact() and dL.guards_intact()
    return dL.host()


@pytest.fixture(params=["single", "pair"])
def cert_kernel(request, monkeypatch):
    """Runs the test with the one-SM certification kernel and with the CTA-pair one."""
    monkeypatch.setenv("GBD_CERT_KERNEL", request.param)
    return request.param


@pytest.mark.parametrize("kind", ["uniform", "e8", "e32", "halves30", "sparse", "blocks", "extreme", "int8"])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
@pytest.mark.parametrize("fp8", [0, 1])
def test_lower_bound_of_abs_product(oracle_mod, kind, ta, tb, fp8, cert_kernel):
    m, n, k = 300, 200, 777  # several tiles and ragged edges in every dimension
    A, lda, B, ldb = _inputs(kind, ta, tb, m, n, k, 500 + len(kind))
    L = _lower_bound(ta, tb, m, n, k, A, lda, B, ldb, fp8)
    G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, 1.0, A, lda, B, ldb, 0.0, None, m)
    # the oracle's G is |A||B| to within a few units in the last place (Dot2 of the magnitudes)
    assert np.all(L <= G * (1.0 + 2.0 ** -50)), first_mismatch(L, G, np.zeros_like(G), m)
    assert np.all(L[G == 0.0] == 0.0)  # a zero |A||B| element has a zero bound
    if not fp8 and kind != "extreme":  # and BF16 planes keep every non-zero one positive
        assert np.all(L[G > 0.0] > 0.0)
    # BF16 planes keep 8 significant bits, E5M2 planes 3 (each factor rounded toward zero)
    tight = {"uniform": (0.97, 0.70), "int8": (0.97, 0.70), "blocks": (0.97, 0.70), "sparse": (0.97, 0.70),
             "halves30": (0.97, None)}.get(kind)
    if tight and tight[fp8]:
        pos = G > 0
        assert np.all(L[pos] >= tight[fp8] * G[pos]), float(np.min(L[pos] / G[pos]))


@pytest.mark.parametrize("k", [16383, 16384 + 64 * 3 + 5])
def test_lower_bound_chunked_inner_dimension(oracle_mod, k, cert_kernel):
    # the one-SM form drains 16384-deep chunks and adds them rounding down; the pair form
    # accumulates the whole inner dimension in TMEM
    m, n = 140, 260
    A = synth.matrix("scaled", k, m, k, 41, 4)
    B = synth.matrix("uniform", k, n, k, 42)
    for fp8, lo in ((0, 0.9), (1, 0.6)):
        L = _lower_bound("T", "N", m, n, k, A, k, B, k, fp8)
        G = oracle_mod.abs_bound_rows("T", "N", m, n, k, 1.0, A, k, B, k, 0.0, None, m)
        assert np.all(L <= G * (1.0 + 2.0 ** -50)) and np.all(L >= lo * G)


def test_lower_bound_nonfinite_rows_and_columns(oracle_mod):
    m, n, k = 130, 140, 150
    A = synth.matrix("uniform", m, k, m, 1)
    B = synth.matrix("uniform", k, n, k, 2)
    A[3 * m + 5] = np.inf  # row 5 of A
    B[7 * k + 4] = np.nan  # column 7 of B
    L = _lower_bound("N", "N", m, n, k, A, m, B, k).reshape(n, m).T
    assert np.isnan(L[5, :]).all() and np.isnan(L[:, 7]).all()
    Lm = np.delete(np.delete(L, 5, axis=0), 7, axis=1)
    assert np.isfinite(Lm).all() and (Lm > 0).all()


def _run(fn, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, prec, tol=0.0):
    import torch
    dA, dB, dC = DeviceBuf(A), DeviceBuf(B), DeviceBuf(C)
    wsb = (gbdgemm.gbd_dgemm_emu_workspace_size if fn == "split" else gbdgemm.gbd_dgemm_emu_mod_workspace_size)(
        m, n, k, prec)
    ws = torch.full((wsb // 8 + 64,), float("nan"), dtype=torch.float64, device="cuda")
    info = gbdgemm.GbdEmuInfo()
    call = gbdgemm.gbd_dgemm_emu if fn == "split" else gbdgemm.gbd_dgemm_emu_mod
    rc = call(ta, tb, m, n, k, alpha, dA.ptr, lda, dB.ptr, ldb, beta, dC.ptr, ldc, prec, tol, ws, wsb, info)
    torch.cuda.synchronize()
    return rc, dC.host(), info


def _check_bound(oracle_mod, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, out, tol):
    ref = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    got = synth.view(out, m, n, ldc).flatten(order="F")
    msg = first_mismatch(got, ref, tol * G, m)
    assert msg is None, msg


@pytest.fixture(params=["fp8", "bf16"])
def cert_dtype(request, monkeypatch):
    """Runs the test with the emulations' FP8 magnitude planes and with BF16 ones."""
    monkeypatch.setenv("GBD_CERT_DTYPE", request.param)
    return request.param


@pytest.mark.parametrize("kind", ["uniform", "e8", "e32", "halves4", "halves8", "sparse", "blocks", "int8", "extreme"])
@pytest.mark.parametrize("tol", [0.0, 1e-10])
def test_modular_choice_matches_the_rule(oracle_mod, kind, tol, cert_dtype):
    m, n, k = 260, 190, 900
    ta, tb = "T", "N"
    A, lda, B, ldb = _inputs(kind, ta, tb, m, n, k, 600 + len(kind))
    C = synth.matrix("uniform", m, n, m, 3)
    c = oracle_mod.certify(ta, tb, m, n, k, A, lda, B, ldb, tol)
    rc, out, info = _run("mod", ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, m, 0, tol)
    if c["moduli"] == 0:  # the rule finds no bit count within 16 moduli
        assert rc == gbdgemm.GBD_ERR_LIMIT
        return
    assert rc == 0, gbdgemm.gbd_last_error()
    assert info.path == gbdgemm.GBD_PATH_MODULAR
    if c["t"] == c["t_exact"] and c["t"] < c["t_cert"]:
        assert info.exact == 1 and info.digit_bits == c["t"]
    else:
        assert c["t"] <= info.digit_bits <= c["t"] + 1, (c, info.digit_bits)
        assert info.rho >= c["rho"] * (1 - 1e-6) and info.gamma >= c["gamma"] * (1 - 1e-6)
    # the moduli: the Cauchy-Schwarz count from upper bounds of the square sums, never more than
    # the k 2^(2t) count and at most one more than the exact square sums give
    n_cs = oracle_mod.cert_moduli_cs(info.digit_bits, k, c["alpha2"], c["beta2"])
    assert n_cs <= info.products <= min(oracle_mod.cert_moduli(info.digit_bits, k), n_cs + 1), (c, info.products)
    _check_bound(oracle_mod, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, m, out, tol if tol > 0 else 2 * k * U)
    model = oracle_mod.ozmod_dgemm_rows(ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, m, info.digit_bits)
    assert first_mismatch(synth.view(out, m, n, m).flatten(order="F"), model, None, m) is None


@pytest.mark.parametrize("kind", ["uniform", "e8", "halves4", "sparse", "blocks", "int8"])
def test_split_choice_matches_the_rule(oracle_mod, kind, cert_dtype):
    m, n, k = 230, 170, 700
    ta, tb = "N", "T"
    A, lda, B, ldb = _inputs(kind, ta, tb, m, n, k, 700 + len(kind))
    C = synth.matrix("uniform", m, n, m, 4)
    c = oracle_mod.certify(ta, tb, m, n, k, A, lda, B, ldb)
    rc, out, info = _run("split", ta, tb, m, n, k, -0.5, A, lda, B, ldb, 2.0, C, m, 0)
    assert rc == 0, gbdgemm.gbd_last_error()
    if c["s"] == c["s_exact"] and c["s"] < c["s_cert"]:
        assert info.exact == 1 and info.slices == c["s"]
    elif c["s"] <= 9:
        assert info.path == gbdgemm.GBD_PATH_SPLIT and c["s"] <= info.slices <= c["s"] + 1, (c, info.slices)
    _check_bound(oracle_mod, ta, tb, m, n, k, -0.5, A, lda, B, ldb, 2.0, C, m, out, 2 * k * U)
    if info.path == gbdgemm.GBD_PATH_SPLIT:
        model = oracle_mod.ozaki_dgemm_rows(ta, tb, m, n, k, -0.5, A, lda, B, ldb, 2.0, C, m, info.slices)
        assert first_mismatch(synth.view(out, m, n, m).flatten(order="F"), model, None, m) is None


def _halves(m, n, k, d=30):
    A = synth.halves_matrix(m, k, m, 901, d, small_cols_from=k // 2)
    B = synth.halves_matrix(k, n, k, 902, d, small_rows_below=k // 2)
    return A, B


def test_structured_input_modular_refuses(oracle_mod):
    import torch
    m = n = 64
    k = 1024
    A, B = _halves(m, n, k)
    C = synth.matrix("uniform", m, n, m, 5)
    rc, out, info = _run("mod", "N", "N", m, n, k, 1.0, A, m, B, k, 0.5, C, m, 0)
    assert rc == gbdgemm.GBD_ERR_LIMIT and "certified" in gbdgemm.gbd_last_error()
    assert np.array_equal(out.view(np.uint64), C.view(np.uint64))  # C untouched
    assert gbdgemm.gbd_check_device_error() == 0
    rc, out, info = _run("mod", "N", "N", m, n, k, 1.0, A, m, B, k, 0.5, C, m, -1)
    assert rc == 0 and gbdgemm.gbd_check_device_error() == gbdgemm.GBD_ERR_LIMIT
    assert np.isnan(out).all()
    torch.cuda.synchronize()


def test_structured_input_split_falls_back(oracle_mod):
    m = n = 64
    k = 1024
    A, B = _halves(m, n, k)
    C = synth.matrix("uniform", m, n, m, 6)
    rc, out, info = _run("split", "N", "N", m, n, k, 1.0, A, m, B, k, 0.5, C, m, 0)
    assert rc == 0, gbdgemm.gbd_last_error()
    assert info.path == gbdgemm.GBD_PATH_NATIVE and info.slices == 0
    _check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, m, B, k, 0.5, C, m, out, 2 * k * U)


def test_structured_input_grouped_falls_back(oracle_mod):
    import ctypes
    import torch
    m = n = 64
    k = 1024
    A, B = _halves(m, n, k)
    A2 = synth.matrix("uniform", m, k, m, 910)
    B2 = synth.matrix("uniform", k, n, k, 911)
    dA, dB, dA2, dB2 = (torch.from_numpy(x).cuda() for x in (A, B, A2, B2))
    dC = torch.zeros(2 * m * n, dtype=torch.float64, device="cuda")
    probs = [dict(transa=b"N", transb=b"N", mode=gbdgemm.GBD_MODE_EMULATED, slices=0, m=m, n=n, k=k, alpha=1.0,
                  beta=0.0, A=a, lda=m, B=b, ldb=k, C=dC[i * m * n:].data_ptr(), ldc=m, tol=0.0)
             for i, (a, b) in enumerate(((dA, dB), (dA2, dB2)))]
    arr = gbdgemm.problem_array(probs)
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    used = (ctypes.c_int * 2)()
    assert gbdgemm.gbd_dgemm_grouped(arr, ws, wsb, used) == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    assert used[0] == -1 and 1 <= used[1] <= 9
    out = dC.cpu().numpy()
    for i, (a, b) in enumerate(((A, B), (A2, B2))):
        ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, a, m, b, k, 0.0, None, m)
        G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.0, a, m, b, k, 0.0, None, m)
        assert first_mismatch(out[i * m * n:(i + 1) * m * n], ref, 2 * k * U * G, m) is None


def test_milder_structure_is_certified(oracle_mod):
    # 2^-8 halves: certifiable, at more bits than uniform data needs, and within the bound
    m = n = 128
    k = 2048
    A, B = _halves(m, n, k, d=8)
    C = synth.matrix("uniform", m, n, m, 7)
    c = oracle_mod.certify("N", "N", m, n, k, A, m, B, k)
    rc, out, info = _run("mod", "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, 0)
    assert rc == 0 and c["t"] <= info.digit_bits <= c["t"] + 1
    _check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, out, 2 * k * U)
    rc, out, info = _run("split", "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, 0)
    assert rc == 0
    _check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, out, 2 * k * U)
