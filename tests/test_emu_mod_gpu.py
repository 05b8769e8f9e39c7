"""GPU parity of the modular emulation (gbd_dgemm_emu_mod) with its CPU model.

The model (oracle/ozaki_mod_model.c) evaluates the exact integer product A'B' directly;
the GPU obtains it from residue products and the Chinese remainder theorem, so equal
bits check the residues, the modular tensor-core products and the reconstruction.  The
automatic mode is checked against the FP64 bound of the Dot2 oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, DeviceBuf, first_mismatch, padding_intact
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def _stored(t, rows, cols):
    return (cols, rows) if t == "T" else (rows, cols)


def _problem(ta, tb, m, n, k, kind, seed, pads=(0, 0, 0), e=0):
    ra, ca = _stored(ta, m, k)
    rb, cb = _stored(tb, k, n)
    lda, ldb, ldc = ra + pads[0], rb + pads[1], m + pads[2]
    A = synth.matrix(kind, ra, ca, lda, seed, e=e)
    B = synth.matrix(kind, rb, cb, ldb, seed + 1, e=e)
    C = synth.matrix("uniform", m, n, ldc, seed + 2)
    return A, lda, B, ldb, C, ldc


def run_mod(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, bits, tol=0.0):
    import torch
    dA, dB, dC = DeviceBuf(A), DeviceBuf(B), DeviceBuf(C)
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(m, n, k, bits)
    ws = torch.full((wsb // 8 + 64,), float("nan"), dtype=torch.float64, device="cuda")  # garbage on entry
    info = gbdgemm.GbdEmuInfo()
    torch.cuda.synchronize()
    rc = gbdgemm.gbd_dgemm_emu_mod(ta, tb, m, n, k, alpha, dA.ptr, lda, dB.ptr, ldb, beta, dC.ptr, ldc, bits, tol,
                                   ws, wsb, info)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0, gbdgemm.gbd_last_error()
    assert dA.guards_intact() and dB.guards_intact() and dC.guards_intact()
    out = dC.host()
    assert padding_intact(out, m, n, ldc)
    return out, info


def check_model(oracle_mod, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, out, bits):
    ref = oracle_mod.ozmod_dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, bits)
    msg = first_mismatch(synth.view(out, m, n, ldc).flatten(order="F"), ref, None, m)
    assert msg is None, msg


@pytest.mark.parametrize("bits", [6, 20, 33, 44])
def test_model_parity_bits(oracle_mod, bits):
    m, n, k = 200, 300, 333
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "scaled", 30 + bits, pads=(3, 1, 2), e=6)
    out, info = run_mod("N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, bits)
    assert info.digit_bits == bits and 1 <= info.slices <= 16
    check_model(oracle_mod, "N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, out, bits)


@pytest.mark.parametrize("kernel", ["single", "pair", "split"])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_model_parity_transposes(oracle_mod, monkeypatch, kernel, ta, tb):
    # the one-SM kernel, the two-SM kernel, and the one-SM kernel with each tile's moduli split
    # over several CTAs (the last to finish rebuilds the tile)
    monkeypatch.setenv("GBD_EMU_KERNEL", kernel)
    m, n, k = 260, 190, 515
    A, lda, B, ldb, C, ldc = _problem(ta, tb, m, n, k, "uniform", 40, pads=(2, 5, 1))
    out, _ = run_mod(ta, tb, m, n, k, -0.75, A, lda, B, ldb, 2.0, C, ldc, 40)
    check_model(oracle_mod, ta, tb, m, n, k, -0.75, A, lda, B, ldb, 2.0, C, ldc, out, 40)


@pytest.mark.parametrize("kernel", ["single", "pair", "split"])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (127, 129, 63), (129, 1, 1025), (33, 257, 65), (5, 3, 70001),
                                   (600, 520, 300)])
def test_model_parity_fringes(oracle_mod, monkeypatch, kernel, m, n, k):
    monkeypatch.setenv("GBD_EMU_KERNEL", kernel)
    # ragged tiles and k-blocks; k > 65536 exercises the periodic reduction of the int32 sums
    A, lda, B, ldb, C, ldc = _problem("T", "N", m, n, k, "uniform", m + n + k, pads=(1, 3, 5))
    out, _ = run_mod("T", "N", m, n, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, 30)
    check_model(oracle_mod, "T", "N", m, n, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, out, 30)


@pytest.mark.parametrize("m,n,k", [(2300, 2310, 100), (700, 300, 1500)])
def test_model_parity_pair_partial_last_wave(oracle_mod, monkeypatch, m, n, k):
    # the two-SM kernel's (tile, modulus) units leave a partial last wave over the SM pairs
    # (9 x 10 tiles of 256 x 256, or 3 x 2, times the moduli); ragged in m, n and k
    monkeypatch.setenv("GBD_EMU_KERNEL", "pair")
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, "uniform", 77 + m, pads=(1, 2, 3))
    out, _ = run_mod("N", "T", m, n, k, 0.5, A, lda, B, ldb, -1.5, C, ldc, 36)
    check_model(oracle_mod, "N", "T", m, n, k, 0.5, A, lda, B, ldb, -1.5, C, ldc, out, 36)


@pytest.mark.parametrize("group_m", ["1", "3", "64"])
def test_model_parity_pair_raster_groups(oracle_mod, monkeypatch, group_m):
    # the raster group height only reorders the pairs' work: the same bits for any of them
    monkeypatch.setenv("GBD_EMU_KERNEL", "pair")
    monkeypatch.setenv("GBD_EMU_GROUP_M", group_m)
    m, n, k = 1300, 1100, 300
    A, lda, B, ldb, C, ldc = _problem("T", "N", m, n, k, "uniform", 91, pads=(2, 1, 4))
    out, _ = run_mod("T", "N", m, n, k, 1.25, A, lda, B, ldb, 0.0, C, ldc, 40)
    check_model(oracle_mod, "T", "N", m, n, k, 1.25, A, lda, B, ldb, 0.0, C, ldc, out, 40)


def test_integer_inputs_bit_exact(oracle_mod):
    m, n, k = 150, 170, 900
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, "int8", 7, pads=(1, 1, 1))
    out, _ = run_mod("N", "T", m, n, k, 2.0, A, lda, B, ldb, -1.0, C, ldc, 20)
    Ai = synth.view(A, m, k, lda).astype(np.int64)
    Bi = synth.view(B, n, k, ldb).astype(np.int64).T
    Ci = synth.view(C, m, n, ldc)
    assert np.array_equal(synth.view(out, m, n, ldc), (2 * (Ai @ Bi)).astype(np.float64) - Ci)


def test_nonfinite_rows_and_columns(oracle_mod):
    m, n, k = 70, 60, 90
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "uniform", 8)
    A[3 + 5 * lda] = np.inf       # row 3
    A[10 + 7 * lda] = np.nan      # row 10
    B[4 + 20 * ldb] = -np.inf     # column 20
    out, _ = run_mod("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc, 25)
    check_model(oracle_mod, "N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.5, C, ldc, out, 25)
    got = synth.view(out, m, n, ldc)
    assert np.isnan(got[3]).all() and np.isnan(got[10]).all() and np.isnan(got[:, 20]).all()


@pytest.mark.parametrize("case", ["near_underflow", "subnormal_results", "overflow"])
def test_model_parity_extreme_exponents(oracle_mod, case):
    m, n, k = 150, 140, 300
    sa, sb, kind = {"near_underflow": (2.0 ** -510, 2.0 ** -510, "int8"),
                    "subnormal_results": (2.0 ** -530, 2.0 ** -505, "uniform"),
                    "overflow": (2.0 ** 520, 2.0 ** 510, "uniform")}[case]
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, kind, 77, pads=(1, 0, 2))
    A = A * sa
    B = B * sb
    out, _ = run_mod("N", "T", m, n, k, 0.7, A, lda, B, ldb, 0.0, C, ldc, 36)
    check_model(oracle_mod, "N", "T", m, n, k, 0.7, A, lda, B, ldb, 0.0, C, ldc, out, 36)


@pytest.mark.parametrize("e", [0, 8])
def test_auto_within_fp64_bound(oracle_mod, e):
    m, n, k = 500, 400, 1200
    A, lda, B, ldb, C, ldc = _problem("T", "N", m, n, k, "scaled", 50 + e, pads=(2, 0, 1), e=e)
    out, info = run_mod("T", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, 0)
    assert 1 <= info.slices <= 16 and info.digit_bits >= 1
    ref = oracle_mod.dgemm_rows("T", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc)
    G = oracle_mod.abs_bound_rows("T", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc)
    got = synth.view(out, m, n, ldc).flatten(order="F")
    assert first_mismatch(got, ref, 2 * k * U * G, m) is None
    check_model(oracle_mod, "T", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, out, info.digit_bits)


def test_auto_large_square_sampled_rows(oracle_mod):
    import torch
    m = n = k = 8192
    A = synth.matrix("uniform", m, k, m, 9000, pad=0.0)
    B = synth.matrix("uniform", k, n, k, 9001, pad=0.0)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(m, n, k, 0)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    info = gbdgemm.GbdEmuInfo()
    rc = gbdgemm.gbd_dgemm_emu_mod("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m, 0, 0.0, ws, wsb, info)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    out = dC.cpu().numpy()
    # 96 seeded rows and the first and last ones, each against the Dot2 oracle's bound
    rows = sorted(set([0, m - 1] + [int(r) for r in synth.splitmix64(9002, 96) % m]))
    ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, rows=rows)
    G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, rows=rows)
    got = out.reshape(n, m)[:, rows].flatten()
    assert first_mismatch(got, ref, 2 * k * U * G, len(rows)) is None
    model = oracle_mod.ozmod_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, info.digit_bits,
                                        rows=rows[:4])
    assert first_mismatch(out.reshape(n, m)[:, rows[:4]].flatten(), model, None, 4) is None


def test_errors_and_quick_returns():
    import torch
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(4, 4, 4, 0)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    call = gbdgemm.gbd_dgemm_emu_mod
    assert call("N", "N", 4, 4, 4, 1.0, z, 4, z, 4, 0.0, z, 4, 63, 0.0, ws, wsb) == gbdgemm.GBD_ERR_ARG
    assert call("N", "N", 4, 4, 4, 1.0, z, 4, z, 4, 0.0, z, 4, -2, 0.0, ws, wsb) == gbdgemm.GBD_ERR_ARG
    # 2 k 2^(2t) = 2^127 at t = 62, k = 4: more than 16 moduli
    assert call("N", "N", 4, 4, 4, 1.0, z, 4, z, 4, 0.0, z, 4, 62, 0.0, ws, wsb) == gbdgemm.GBD_ERR_LIMIT
    # an accuracy target beyond 16 moduli in automatic mode
    o = torch.ones(64, dtype=torch.float64, device="cuda")
    assert call("N", "N", 4, 4, 4, 1.0, o, 4, o, 4, 0.0, z, 4, 0, 1e-40, ws, wsb) == gbdgemm.GBD_ERR_LIMIT
    assert call("N", "N", 4, 4, 4, 1.0, z, 4, z, 4, 0.0, z, 4, 10, 0.0, ws, 64) == gbdgemm.GBD_ERR_WORKSPACE
    assert call("N", "N", 4, 4, 4, 1.0, z, 3, z, 4, 0.0, z, 4, 10, 0.0, ws, wsb) == 8
    C = torch.arange(16, dtype=torch.float64, device="cuda")
    assert call("N", "N", 4, 4, 0, 1.0, z, 4, z, 1, 3.0, C, 4, 0, 0.0, ws, wsb) == 0
    torch.cuda.synchronize()
    assert torch.equal(C, 3.0 * torch.arange(16, dtype=torch.float64, device="cuda"))


def test_deterministic():
    m, n, k = 300, 280, 2000
    A, lda, B, ldb, C, ldc = _problem("N", "N", m, n, k, "scaled", 3, e=8)
    o1, i1 = run_mod("N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, 0)
    o2, i2 = run_mod("N", "N", m, n, k, 1.5, A, lda, B, ldb, -0.5, C, ldc, 0)
    assert np.array_equal(o1.view(np.uint64), o2.view(np.uint64)) and i1.digit_bits == i2.digit_bits


@pytest.mark.parametrize("m,n,k", [(2048, 2048, 256), (4096, 4096, 256)])
def test_kernel_launches_per_call(m, n, k):
    # one call with the bits chosen on the device launches the kernels that the benchmark's
    # launch count claims (preparation, certification, plans, residues, column scales, products,
    # reconstruction)
    import torch
    from torch.profiler import ProfilerActivity, profile

    import bench
    A = torch.rand(m * k, dtype=torch.float64, device="cuda") - 0.5
    B = torch.rand(k * n, dtype=torch.float64, device="cuda") - 0.5
    C = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(m, n, k, -1)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")

    def call():
        rc = gbdgemm.gbd_dgemm_emu_mod("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, -1, 0.0, ws, wsb, None)
        assert rc == 0, gbdgemm.gbd_last_error()

    call()
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]):  # the profiler's own first use
        C.add_(0.0)
        torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        call()
        torch.cuda.synchronize()
    names = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA]
    kernels = [x for x in names if "k_" in x and ("emu::" in x or "gbd::" in x)]
    if not names:
        pytest.skip("the profiler recorded no device activity here")
    assert len(kernels) == bench.MOD_LAUNCHES, kernels
    assert gbdgemm.gbd_check_device_error() == 0


@pytest.mark.parametrize("e", [0, 8])
def test_device_side_automatic_mode_matches_the_synchronising_one(oracle_mod, e):
    # bits = -1 chooses on the device exactly as bits = 0 does, without any read-back
    m, n, k = 400, 300, 900
    A, lda, B, ldb, C, ldc = _problem("N", "T", m, n, k, "scaled", 60 + e, pads=(1, 2, 3), e=e)
    out0, info0 = run_mod("N", "T", m, n, k, 1.25, A, lda, B, ldb, -0.75, C, ldc, 0)
    out1, info1 = run_mod("N", "T", m, n, k, 1.25, A, lda, B, ldb, -0.75, C, ldc, -1)
    assert np.array_equal(out0.view(np.uint64), out1.view(np.uint64))
    assert (info1.digit_bits, info1.products, info1.bound) == (info0.digit_bits, info0.products, info0.bound)
    check_model(oracle_mod, "N", "T", m, n, k, 1.25, A, lda, B, ldb, -0.75, C, ldc, out1, info1.digit_bits)


def test_device_side_automatic_mode_unreachable_target():
    # a target beyond 16 moduli: C becomes NaN, the device error word reports GBD_ERR_LIMIT,
    # and the synchronising form refuses before touching C
    import torch
    m = n = k = 64
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(m, n, k, 0)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    A = torch.ones(m * k, dtype=torch.float64, device="cuda")
    C = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    assert gbdgemm.gbd_dgemm_emu_mod("N", "N", m, n, k, 1.0, A, m, A, k, 0.0, C, m, 0, 1e-40, ws, wsb) == \
        gbdgemm.GBD_ERR_LIMIT
    torch.cuda.synchronize()
    assert torch.count_nonzero(C).item() == 0 and gbdgemm.gbd_check_device_error() == 0
    assert gbdgemm.gbd_dgemm_emu_mod("N", "N", m, n, k, 1.0, A, m, A, k, 0.0, C, m, -1, 1e-40, ws, wsb) == 0
    assert gbdgemm.gbd_check_device_error() == gbdgemm.GBD_ERR_LIMIT
    assert torch.isnan(C).all().item()
    assert gbdgemm.gbd_check_device_error() == 0  # read and cleared


@pytest.mark.parametrize("bits", [0, -1])
def test_split_form_repeated_calls_reuse_counters(oracle_mod, monkeypatch, bits):
    # the split form's per-tile counters are cleared by every call: three calls on one workspace agree
    import torch
    monkeypatch.setenv("GBD_EMU_KERNEL", "split")
    m, n, k = 300, 260, 700
    A, lda, B, ldb, C, ldc = _problem("T", "T", m, n, k, "uniform", 88, pads=(1, 1, 1))
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(m, n, k, bits)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    outs = []
    for _ in range(3):
        dC = torch.from_numpy(C).cuda()
        info = gbdgemm.GbdEmuInfo()
        assert gbdgemm.gbd_dgemm_emu_mod("T", "T", m, n, k, 0.5, dA, lda, dB, ldb, 1.5, dC, ldc, bits, 0.0, ws, wsb,
                                         info) == 0
        torch.cuda.synchronize()
        assert gbdgemm.gbd_check_device_error() == 0
        outs.append(dC.cpu().numpy())
    assert all(np.array_equal(outs[0].view(np.uint64), o.view(np.uint64)) for o in outs[1:])
    check_model(oracle_mod, "T", "T", m, n, k, 0.5, A, lda, B, ldb, 1.5, C, ldc, outs[0], info.digit_bits)
