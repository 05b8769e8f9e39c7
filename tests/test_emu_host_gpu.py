"""gbd_dgemm_emu_host: the emulated DGEMM on operands in host memory.

Checks: the result is the same bits as gbd_dgemm_emu on device copies with the
same slice count, and within the oracle's FP64 bound; the leading-dimension
padding of the host C is neither read nor written; pinned (host tensors) and
pageable (numpy) memory; the quick returns; a buffer that is too small; and two
calls in flight on two streams with two buffers.
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, first_mismatch, padding_intact
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def _operands(seed, m, n, k, ta, tb, pad):
    ra, ca = (k, m) if ta == "T" else (m, k)
    rb, cb = (n, k) if tb == "T" else (k, n)
    lda, ldb, ldc = ra + pad, rb + 2 * pad, m + pad
    A = synth.matrix("uniform", ra, ca, lda, seed)
    B = synth.matrix("scaled", rb, cb, ldb, seed + 1, e=8)
    C = synth.matrix("uniform", m, n, ldc, seed + 2)
    return A, lda, B, ldb, C, ldc


def _device_reference(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices):
    import torch
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
    wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, slices)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    gbdgemm.check(gbdgemm.gbd_dgemm_emu(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, slices, 0.0,
                                        ws, wsb))
    torch.cuda.synchronize()
    return synth.view(dC.cpu().numpy(), m, n, ldc)


def _call_host(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, stream=None):
    import torch
    size = gbdgemm.gbd_dgemm_emu_host_buffer_size(ta, tb, m, n, k, slices)
    buf = torch.empty(max(size, 1), dtype=torch.uint8, device="cuda")
    info = gbdgemm.GbdEmuInfo()
    rc = gbdgemm.gbd_dgemm_emu_host(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, 0.0, buf, size,
                                    info, stream=stream)
    return rc, info, buf


@pytest.mark.parametrize("m,n,k,ta,tb,alpha,beta,pinned", [
    (300, 257, 199, "N", "N", 1.5, -0.5, True),
    (129, 400, 1000, "T", "N", -1.0, 0.0, False),
    (200, 133, 517, "N", "T", 0.75, 2.0, True),
    (64, 64, 2049, "T", "T", 1.0, 1.0, False),
])
def test_same_bits_as_the_device_call(oracle_mod, m, n, k, ta, tb, alpha, beta, pinned):
    import torch
    A, lda, B, ldb, C0, ldc = _operands(900 + m, m, n, k, ta, tb, pad=3)
    C = C0.copy()
    if pinned:
        At, Bt, Ct = (torch.from_numpy(x).pin_memory() for x in (A, B, C))
        rc, info, _ = _call_host(ta, tb, m, n, k, alpha, At, lda, Bt, ldb, beta, Ct, ldc, 0)
        torch.cuda.synchronize()
        C = Ct.numpy()
    else:
        rc, info, _ = _call_host(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0)
        torch.cuda.synchronize()
    assert rc == 0, gbdgemm.gbd_last_error()
    assert padding_intact(C, m, n, ldc)  # the sentinel padding of C is untouched
    got = synth.view(C, m, n, ldc)
    ref = _device_reference(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, info.slices)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    exact = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    assert first_mismatch(got.flatten(order="F"), exact, 2 * k * U * G, m) is None


def test_quick_returns():
    import torch
    m, n, k = 33, 17, 40
    A, lda, B, ldb, C0, ldc = _operands(5, m, n, k, "N", "N", pad=2)
    for alpha, kk in ((0.0, k), (1.0, 0)):
        C = C0.copy()
        rc, _, _ = _call_host("N", "N", m, n, kk, alpha, A, lda, B, ldb, -2.0, C, ldc, 0)
        torch.cuda.synchronize()
        assert rc == 0, gbdgemm.gbd_last_error()
        assert np.array_equal(synth.view(C, m, n, ldc), -2.0 * synth.view(C0, m, n, ldc))
        assert padding_intact(C, m, n, ldc)


def test_buffer_too_small_is_refused():
    import torch
    m = n = k = 64
    A, lda, B, ldb, C, ldc = _operands(6, m, n, k, "N", "N", pad=0)
    size = gbdgemm.gbd_dgemm_emu_host_buffer_size("N", "N", m, n, k, 0)
    buf = torch.empty(size, dtype=torch.uint8, device="cuda")
    rc = gbdgemm.gbd_dgemm_emu_host("N", "N", m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, 0, 0.0, buf, size - 256)
    assert rc == gbdgemm.GBD_ERR_WORKSPACE


def test_two_streams_in_flight():
    import torch
    m, n, k = 384, 320, 700
    jobs = []
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    keep = []
    for i in range(4):
        A, lda, B, ldb, C0, ldc = _operands(40 + i, m, n, k, "N", "T", pad=1)
        At, Bt, Ct = (torch.from_numpy(x).pin_memory() for x in (A, B, C0.copy()))
        rc, info, buf = _call_host("N", "T", m, n, k, 1.0, At, lda, Bt, ldb, 0.5, Ct, ldc, 6,
                                   stream=streams[i % 2])
        assert rc == 0, gbdgemm.gbd_last_error()
        keep += [buf, At, Bt]  # the buffers stay alive until the copies have run
        jobs.append((A, lda, B, ldb, C0, ldc, Ct))
    torch.cuda.synchronize()
    for A, lda, B, ldb, C0, ldc, Ct in jobs:
        ref = _device_reference("N", "T", m, n, k, 1.0, A, lda, B, ldb, 0.5, C0, ldc, 6)
        assert np.array_equal(synth.view(Ct.numpy(), m, n, ldc).view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("m,n,k,ta,tb,alpha,beta,bits,pinned", [
    (300, 257, 199, "N", "N", 1.5, -0.5, 0, True),
    (129, 400, 1000, "T", "N", -1.0, 0.0, 40, False),
    (200, 133, 517, "N", "T", 0.75, 2.0, 0, False),
])
def test_modular_host_call_matches_the_model(oracle_mod, m, n, k, ta, tb, alpha, beta, bits, pinned):
    import torch
    A, lda, B, ldb, C0, ldc = _operands(950 + m, m, n, k, ta, tb, pad=3)
    C = C0.copy()
    hA, hB, hC = (torch.from_numpy(x) for x in (A, B, C))
    if pinned:
        hA, hB, hC = hA.pin_memory(), hB.pin_memory(), hC.pin_memory()
    size = gbdgemm.gbd_dgemm_emu_mod_host_buffer_size(ta, tb, m, n, k, bits)
    buf = torch.empty(size, dtype=torch.uint8, device="cuda")
    info = gbdgemm.GbdEmuInfo()
    rc = gbdgemm.gbd_dgemm_emu_mod_host(ta, tb, m, n, k, alpha, hA, lda, hB, ldb, beta, hC, ldc, bits, 0.0, buf, size,
                                        info)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    out = hC.numpy()
    assert padding_intact(out, m, n, ldc)
    assert bits == 0 or info.digit_bits == bits
    ref = oracle_mod.ozmod_dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, info.digit_bits)
    assert first_mismatch(synth.view(out, m, n, ldc).flatten(order="F"), ref, None, m) is None
    if bits == 0:
        G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
        want = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
        assert first_mismatch(synth.view(out, m, n, ldc).flatten(order="F"), want, 2 * k * U * G, m) is None
    assert gbdgemm.gbd_dgemm_emu_mod_host(ta, tb, m, n, k, alpha, hA, lda, hB, ldb, beta, hC, ldc, bits, 0.0, buf,
                                          64) == gbdgemm.GBD_ERR_WORKSPACE
