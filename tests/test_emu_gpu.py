"""Parity of the split emulation (gbd_dgemm_emu) on the tcgen05 tensor cores.

Two oracles: (1) the CPU model of the same method (oracle/ozaki_model.c), which
must agree bit for bit because every integer level sum is exact on both sides
and the FP64 updates run in the same order; (2) the plain Dot2 oracle, against
which the automatic slice count must meet the componentwise FP64 bound
|C - C_oracle| <= 2 k u G (bit-exact on small-integer inputs).
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, DeviceBuf, first_mismatch, padding_intact
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def _stored(trans, rows, cols):
    return (cols, rows) if trans in "TtCc" else (rows, cols)


def run_emu(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, tol=0.0, stream=None):
    import torch
    dA, dB, dC = DeviceBuf(A), DeviceBuf(B), DeviceBuf(C)
    wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, slices)
    ws = torch.full((wsb // 8 + 64,), float("nan"), dtype=torch.float64, device="cuda")  # garbage on entry
    info = gbdgemm.GbdEmuInfo()
    torch.cuda.synchronize()
    rc = gbdgemm.gbd_dgemm_emu(ta, tb, m, n, k, alpha, dA.ptr, lda, dB.ptr, ldb, beta, dC.ptr, ldc, slices, tol,
                               ws, wsb, info, stream=stream)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0, gbdgemm.gbd_last_error()
    assert dA.guards_intact() and dB.guards_intact() and dC.guards_intact()
    out = dC.host()
    assert padding_intact(out, m, n, ldc)
    return out, info


def _problem(ta, tb, m, n, k, kind, seed, pads=(0, 0, 0), e=0, ckind="uniform"):
    ra, ca = _stored(ta, m, k)
    rb, cb = _stored(tb, k, n)
    lda, ldb, ldc = ra + pads[0], rb + pads[1], m + pads[2]
    A = synth.matrix(kind, ra, ca, lda, seed, e=e)
    B = synth.matrix(kind, rb, cb, ldb, seed + 1, e=e)
    C = synth.matrix(ckind, m, n, ldc, seed + 2)
    return A, lda, B, ldb, C, ldc


def _compact(C, m, n, ldc):
    return np.ascontiguousarray(synth.view(C, m, n, ldc)).flatten(order="F")


def check_model(oracle_mod, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, out, slices):
    ref = oracle_mod.ozaki_dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices)
    msg = first_mismatch(_compact(out, m, n, ldc), ref, None, m)
    assert msg is None, msg


def check_bound(oracle_mod, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, out, rows=None, exact=False):
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


# --- the smallest case first: one tile, one slice, integer inputs ---
def test_single_tile_one_slice_integers(oracle_mod):
    m, n, k = 128, 256, 64
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "int8", 1)
    out, info = run_emu("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, slices=1)
    assert info.slices == 1 and info.products == 1
    check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out, exact=True)


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (128, 256, 256), (256, 512, 320), (300, 200, 100)])
def test_tiles_integers_bit_exact(oracle_mod, m, n, k):
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "int8", m + n + k)
    out, _ = run_emu("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, slices=2)
    check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out, exact=True)


# --- bit-exact against the CPU model of the method ---
@pytest.fixture(params=["single", "pair"])
def kernel(request, monkeypatch):
    """Runs the test once with the one-SM slice kernel and once with the two-SM (cta_group::2) one."""
    monkeypatch.setenv("GBD_EMU_KERNEL", request.param)
    return request.param


@pytest.mark.parametrize("slices", [1, 2, 3, 5, 7, 9])
def test_model_parity_slices(oracle_mod, slices, kernel):
    m, n, k = 200, 300, 333
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "scaled", 10 + slices, pads=(3, 1, 2), e=6)
    out, info = run_emu("N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, slices=slices)
    assert info.slices == slices
    check_model(oracle_mod, "N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, out, slices)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_model_parity_transposes(oracle_mod, ta, tb, kernel):
    m, n, k = 257, 129, 515
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "uniform", 40, pads=(8, 8, 8))
    out, _ = run_emu(ta, tb, m, n, k, -1.25, A, lda, B, ldb, 0.75, C, ldc, slices=6)
    check_model(oracle_mod, ta, tb, m, n, k, -1.25, A, lda, B, ldb, 0.75, C, ldc, out, 6)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 3, 7), (127, 129, 63), (129, 255, 65), (64, 700, 1000),
                                   (1000, 33, 129)])
def test_model_parity_fringes(oracle_mod, m, n, k, kernel):
    A, lda, B, ldb, C, ldc = _problem("T", "N", m, n, k, "uniform", m * 3 + n + k, pads=(1, 3, 5))
    out, _ = run_emu("T", "N", m, n, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, slices=4)
    check_model(oracle_mod, "T", "N", m, n, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, out, 4)


def test_model_parity_two_k_segments(oracle_mod, kernel):
    # k > 8192: every level is summed in two integer segments
    m, n, k = 130, 140, 8192 + 200
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, "uniform", 77)
    out, _ = run_emu("N", "T", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, slices=3)
    check_model(oracle_mod, "N", "T", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out, 3)


def test_adversarial_exact_accumulation(oracle_mod, kernel):
    # every digit of every entry is +127 or -127, one sign per half of k: each 1024-deep FP32 chunk
    # sums to 1024 * 127^2 = 16516096 (< 2^24), the largest the method allows; any inexact
    # tensor-core accumulation shows as a mismatch with the exact model
    m, n, k = 128, 256, 2048
    x = 1.0 - 2.0 ** -53  # binary 0.111...1: every 7-bit digit is 127
    A = np.full(m * k, x)
    A[: m * k // 2] = -x
    B = np.full(k * n, x)
    C = np.zeros(m * n)
    out, _ = run_emu("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, slices=7)
    check_model(oracle_mod, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, out, 7)
    # mixed magnitudes: one large product and many +-1 products in the same chunk
    A = synth.matrix("int8", m, k, m, 5, pad=0.0)
    A[:m] = 127.0
    B = synth.matrix("int8", k, n, k, 6, pad=0.0)
    B.reshape(n, k)[:, 0] = 127.0
    out, _ = run_emu("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, slices=1)
    check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, out, exact=True)


@pytest.mark.parametrize("case", ["near_underflow", "subnormal_results", "subnormal_inputs", "overflow"])
def test_model_parity_extreme_exponents(oracle_mod, kernel, case):
    # The level scale is applied as alpha 2^(tau_j - 7h) times Y 2^sigma_i, on both sides; these
    # ranges put results near the underflow threshold, below it, inputs below it, and results
    # past the overflow threshold (Inf).
    m, n, k = 150, 140, 300
    scale_a, scale_b, kind, slices = {
        "near_underflow": (2.0 ** -510, 2.0 ** -510, "int8", 3),
        "subnormal_results": (2.0 ** -530, 2.0 ** -505, "uniform", 9),
        "subnormal_inputs": (2.0 ** -1060, 2.0 ** -10, "uniform", 9),
        "overflow": (2.0 ** 520, 2.0 ** 510, "uniform", 5),
    }[case]
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, kind, 77, pads=(1, 0, 2))
    A = A * scale_a
    B = B * scale_b
    out, _ = run_emu("N", "T", m, n, k, 0.7, A, lda, B, ldb, 0.0, C, ldc, slices=slices)
    check_model(oracle_mod, "N", "T", m, n, k, 0.7, A, lda, B, ldb, 0.0, C, ldc, out, slices)
    got = synth.view(out, m, n, ldc)
    if case == "overflow":
        assert np.isinf(got).any()
    if case in ("subnormal_results", "subnormal_inputs"):
        assert ((got != 0) & (np.abs(got) < 2.0 ** -1022)).any()


@pytest.mark.parametrize("m,n,k", [(200, 150, 20000), (130, 96, 8192 + 130), (64, 64, 1000)])
def test_split_inner_dimension_matches_model(oracle_mod, m, n, k):
    # few output tiles and a deep inner dimension: the one-SM kernel cuts each 8192-deep segment
    # of a tile into sub-ranges whose exact group sums are added as integers; the result must be
    # the model's bits (several segments, a short last segment, uneven sub-ranges)
    A, lda, B, ldb, C, ldc = _problem("T", "N", m, n, k, "scaled", 91, pads=(1, 2, 3), e=5)
    out, info = run_emu("T", "N", m, n, k, -1.25, A, lda, B, ldb, 0.5, C, ldc, slices=7)
    check_model(oracle_mod, "T", "N", m, n, k, -1.25, A, lda, B, ldb, 0.5, C, ldc, out, 7)


def test_nonfinite_rows_and_columns(oracle_mod, kernel):
    m, n, k = 140, 150, 90
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "uniform", 9)
    A[5 * lda + 7] = np.inf     # row 7 of op(A)
    B[11 * ldb + 3] = np.nan    # column 11 of op(B)
    out, _ = run_emu("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, slices=4)
    check_model(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out, 4)
    o = _compact(out, m, n, ldc).reshape(n, m).T
    assert np.isnan(o[7, :]).all() and np.isnan(o[:, 11]).all()


# --- the automatic slice count against the FP64 bound of the plain oracle ---
def test_auto_square_256(oracle_mod):
    m = n = k = 256
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "uniform", synth.seed_for(0))
    out, info = run_emu("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, slices=0)
    assert 1 <= info.slices <= 9 and info.path == gbdgemm.GBD_PATH_SPLIT and info.bound <= 2 * k * U
    check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out)
    check_model(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out, info.slices)


def test_auto_square_256_integers_bit_exact(oracle_mod):
    m = n = k = 256
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "int8", synth.seed_for(0, 1))
    out, info = run_emu("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, slices=0)
    check_bound(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, out, exact=True)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_auto_padded_ld_all_transposes(oracle_mod, ta, tb):
    m, n, k = 1000, 1200, 800
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "uniform", synth.seed_for(1), pads=(8, 8, 8))
    out, info = run_emu(ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, slices=0)
    check_bound(oracle_mod, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, out)


@pytest.mark.parametrize("e", [0, 8, 32])
def test_auto_large_square_sampled_rows(oracle_mod, e):
    import torch
    m = n = k = 8192
    A = synth.matrix("scaled", m, k, m, synth.seed_for(2, e), e=e, pad=0.0)
    B = synth.matrix("scaled", k, n, k, synth.seed_for(2, e) + 1, e=e, pad=0.0)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty(m * n, dtype=torch.float64, device="cuda")
    wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, 0)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    info = gbdgemm.GbdEmuInfo()
    rc = gbdgemm.gbd_dgemm_emu("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, 0, 0.0, ws, wsb, info)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    rows = sorted(set([0, m - 1] + [int(x) for x in synth.splitmix64(synth.seed_for(2, e) + 7, 24) % m]))
    got = dC.view(n, m)[:, rows].t().cpu().numpy().flatten(order="F")
    ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, rows=rows)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, rows=rows)
    msg = first_mismatch(got, ref, 2 * k * U * G, len(rows))
    assert msg is None, f"slices={info.slices}: {msg}"
    if info.path == gbdgemm.GBD_PATH_NATIVE:  # no slice count certified: computed on the FP64 path
        return
    # and bit for bit against the model of the method on two of the rows
    mrows = rows[:2]
    mref = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, info.slices, rows=mrows)
    mgot = dC.view(n, m)[:, mrows].t().cpu().numpy().flatten(order="F")
    assert first_mismatch(mgot, mref, None, len(mrows)) is None


# --- BLAS conventions and errors ---
def test_quick_returns_and_errors():
    import torch
    m, n, k = 40, 30, 20
    nanA = np.full(m * k, np.nan)
    nanB = np.full(k * n, np.nan)
    C = synth.uniform_pm1(1, m * n)
    out, _ = run_emu("N", "N", m, n, k, 0.0, nanA, m, nanB, k, -2.0, C, m, slices=3)
    assert np.array_equal(out, -2.0 * C)
    out, _ = run_emu("N", "N", m, n, 0, 1.0, nanA, m, nanB, 1, 0.5, C, m, slices=0)
    assert np.array_equal(out, 0.5 * C)
    A = synth.uniform_pm1(2, m * k)
    B = synth.uniform_pm1(3, k * n)
    out, _ = run_emu("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, np.full(m * n, np.nan), m, slices=3)
    assert np.isfinite(out).all()
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
    wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, 3)
    ws = torch.empty(wsb + 512, dtype=torch.uint8, device="cuda")
    assert gbdgemm.gbd_dgemm_emu("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, 3, 0.0, ws, wsb - 1) == \
        gbdgemm.GBD_ERR_WORKSPACE
    assert gbdgemm.gbd_dgemm_emu("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, 3, 0.0,
                                 ws.data_ptr() + 8, wsb) == gbdgemm.GBD_ERR_WORKSPACE
    assert gbdgemm.gbd_dgemm_emu("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, 10, 0.0, ws, wsb) == \
        gbdgemm.GBD_ERR_ARG
    assert gbdgemm.gbd_dgemm_emu("N", "N", m, n, k, 1.0, dA, m - 1, dB, k, 0.0, dC, m, 3, 0.0, ws, wsb) == 8


def test_pair_and_single_kernels_agree(monkeypatch):
    m, n, k = 700, 900, 1300
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, "scaled", 8, e=20)
    monkeypatch.setenv("GBD_EMU_KERNEL", "single")
    o1, _ = run_emu("N", "T", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, slices=8)
    monkeypatch.setenv("GBD_EMU_KERNEL", "pair")
    o2, _ = run_emu("N", "T", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, slices=8)
    assert np.array_equal(o1.view(np.uint64), o2.view(np.uint64))


def test_concurrent_host_threads_and_streams():
    # two host threads, each with its own stream, workspace and output, calling the emulated
    # entry point at the same time (ctypes releases the interpreter lock during the call)
    import threading

    import torch
    jobs = []
    for i, (m, n, k) in enumerate([(300, 200, 700), (257, 333, 1500)]):
        A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, "uniform", 60 + i)
        ref, _ = run_emu("N", "T", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc, slices=0)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, 0)
        jobs.append(dict(args=(m, n, k, dA, lda, dB, ldb, C, ldc), ref=ref, wsb=wsb,
                         ws=torch.empty(wsb, dtype=torch.uint8, device="cuda"), stream=torch.cuda.Stream()))
    torch.cuda.synchronize()
    errors = []

    def worker(jb):
        m, n, k, dA, lda, dB, ldb, C, ldc = jb["args"]
        try:
            for _ in range(20):
                dC = torch.from_numpy(C).cuda()
                rc = gbdgemm.gbd_dgemm_emu("N", "T", m, n, k, 1.0, dA, lda, dB, ldb, 0.5, dC, ldc, 0, 0.0, jb["ws"],
                                           jb["wsb"], None, stream=jb["stream"])
                if rc != 0:
                    errors.append(gbdgemm.gbd_last_error())
                    return
                jb["stream"].synchronize()
                if not np.array_equal(dC.cpu().numpy().view(np.uint64), jb["ref"].view(np.uint64)):
                    errors.append("result differs from the single-threaded call")
                    return
        except Exception as exc:  # noqa: BLE001 -- reported to the main thread
            errors.append(repr(exc))

    threads = [threading.Thread(target=worker, args=(jb,)) for jb in jobs]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert gbdgemm.gbd_check_device_error() == 0


def test_deterministic():
    m, n, k = 600, 500, 700
    A, lda, B, ldb, C, ldc = _problem("T", "T", m, n, k, "scaled", 3, e=8)
    o1, _ = run_emu("T", "T", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, slices=8)
    o2, _ = run_emu("T", "T", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, slices=8)
    assert np.array_equal(o1.view(np.uint64), o2.view(np.uint64))


def test_automatic_statistics_do_not_depend_on_block_order():
    # k > 1024: every row's magnitude sum adds several blocks' partial sums; they are added as
    # fixed-point integers, so the statistics behind the automatic slice count repeat exactly
    m, n, k = 300, 260, 5000
    for ta, tb in (("N", "N"), ("T", "T")):
        A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "scaled", 5, e=4)
        infos = [run_emu(ta, tb, m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, slices=0)[1] for _ in range(4)]
        assert len({(i.rho, i.gamma, i.bound, i.slices, i.path) for i in infos}) == 1
