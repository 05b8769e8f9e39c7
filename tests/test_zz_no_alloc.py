"""gbd_dgemm_emu_noalloc: the emulated DGEMM for callers that cannot allocate device memory.

Such callers (latency-critical loops, plug-ins whose host owns all device memory,
code holding an allocator lock) get the same computation with a scratch area
built into the library.  The tests call the entry point through the C ABI several
times in a row on different inputs (each call finds the previous call's contents
in the shared scratch, once with the same shape as an earlier call) and check each
result against the workspace-taking gbd_dgemm_emu: the same slice count must give
the same bits, and both must meet the FP64 bound of the oracle.  They also check
the documented limit (768^3 fits, 769^3 does not) and that a quick return needs no
scratch.  This file is collected last so that a run that
stops at its first failure has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def _problem(seed, m, n, k, ta, tb):
    ra, ca = (k, m) if ta == "T" else (m, k)
    rb, cb = (n, k) if tb == "T" else (k, n)
    A = synth.matrix("uniform", ra, ca, ra + 2, seed, pad=0.0)
    B = synth.matrix("scaled", rb, cb, rb, seed + 1, e=8, pad=0.0)
    C = synth.matrix("uniform", m, n, m + 1, seed + 2, pad=0.0)
    return A, ra + 2, B, rb, C, m + 1


def _with_workspace(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, C, ldc, slices):
    import torch
    dC = torch.from_numpy(C).cuda()
    wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, slices)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    rc = gbdgemm.gbd_dgemm_emu(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, slices, 0.0, ws, wsb)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def _noalloc_and_check(oracle_mod, m, n, k, ta, tb, alpha, beta, slices, seed):
    import torch
    A, lda, B, ldb, C, ldc = _problem(seed, m, n, k, ta, tb)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.from_numpy(C).cuda()
    info = gbdgemm.GbdEmuInfo()
    torch.cuda.synchronize()
    rc = gbdgemm.gbd_dgemm_emu_noalloc(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, slices, 0.0, info)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    got = dC.cpu().numpy()
    used = info.slices
    assert info.path == gbdgemm.GBD_PATH_SPLIT and 1 <= used <= 9 and (slices == 0 or used == slices)
    ref = _with_workspace(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, C, ldc, used)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    exact = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
    mine = synth.view(got, m, n, ldc).flatten(order="F")
    assert first_mismatch(mine, exact, 2 * k * U * G, m) is None
    return used


def test_calls_in_a_row_match_the_workspace_variant(oracle_mod):
    # automatic slices, then an explicit count large enough for the FP64 bound on this data, then
    # the first shape and slice count again on new data: its counters and parked sums fall where
    # the first call left its own, so a missed reset would show
    cases = [(301, 257, 199, "N", "T", 1.5, -0.5, 0, 700), (200, 333, 517, "T", "N", -1.0, 0.0, 9, 710)]
    used = [_noalloc_and_check(oracle_mod, *c) for c in cases]
    m, n, k, ta, tb, alpha, beta, _, _ = cases[0]
    _noalloc_and_check(oracle_mod, m, n, k, ta, tb, alpha, beta, used[0], 720)


def test_largest_square_problem_fits():
    # 768^3 with automatic slices fits the 64 MiB scratch and gives the workspace variant's bits
    import torch
    m = n = k = 768
    assert gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, 0) <= 64 << 20
    A, lda, B, ldb, C, ldc = _problem(730, m, n, k, "N", "N")
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
    info = gbdgemm.GbdEmuInfo()
    rc = gbdgemm.gbd_dgemm_emu_noalloc("N", "N", m, n, k, 1.0, dA, lda, dB, ldb, 0.5, dC, ldc, 0, 0.0, info)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    ref = _with_workspace("N", "N", m, n, k, 1.0, dA, lda, dB, ldb, 0.5, C, ldc, info.slices)
    assert np.array_equal(dC.cpu().numpy().view(np.uint64), ref.view(np.uint64))


def test_quick_return_needs_no_scratch():
    # alpha = 0 at 4096^3: C := beta C, A and B not read, although the product would not fit
    import torch
    m = n = k = 4096
    C0 = torch.arange(m * n, dtype=torch.float64, device="cuda") % 97.0
    C = C0.clone()
    rc = gbdgemm.gbd_dgemm_emu_noalloc("N", "N", m, n, k, 0.0, 0, m, 0, k, -0.5, C, m, 0, 0.0)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert torch.equal(C, -0.5 * C0)


@pytest.mark.parametrize("size", [769, 4096])
def test_problem_above_the_scratch_size_is_refused(size):
    import torch
    m = n = k = size
    rc = gbdgemm.gbd_dgemm_emu_noalloc("N", "N", m, n, k, 1.0, 0, m, 0, k, 0.0, 0, m, 0, 0.0,
                                       stream=torch.cuda.current_stream())
    assert rc == gbdgemm.GBD_ERR_LIMIT
    assert "scratch" in gbdgemm.gbd_last_error()
