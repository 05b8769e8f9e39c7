"""GPU tests of the library context (gbd_create / gbd_ctx_dgemm / gbd_sync_error).

A context call gives the bits of the matching entry point with a caller workspace; the
automatic method takes the modular emulation, the split one when 16 moduli cannot certify
the target, and the FP64 path when 9 slices cannot either; the pool keeps one workspace per
stream and grows it in stream order.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx():
    rc, c = gbdgemm.gbd_create(0)
    assert rc == 0, gbdgemm.gbd_last_error()
    yield c
    gbdgemm.gbd_destroy(c)


def _dev(*arrs):
    import torch
    return [torch.from_numpy(a).cuda() for a in arrs]


def _direct(method, ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, C0, ldc):
    import torch
    dC = torch.from_numpy(C0).cuda()
    if method == gbdgemm.GBD_METHOD_NATIVE:
        gbdgemm.check(gbdgemm.gbd_dgemm(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc))
    else:
        split = method == gbdgemm.GBD_METHOD_SPLIT
        size = gbdgemm.gbd_dgemm_emu_workspace_size if split else gbdgemm.gbd_dgemm_emu_mod_workspace_size
        wsb = size(m, n, k, 0)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        call = gbdgemm.gbd_dgemm_emu if split else gbdgemm.gbd_dgemm_emu_mod
        gbdgemm.check(call(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, 0, 0.0, ws, wsb))
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("method", [gbdgemm.GBD_METHOD_NATIVE, gbdgemm.GBD_METHOD_SPLIT, gbdgemm.GBD_METHOD_MODULAR])
def test_context_call_matches_the_entry_point(ctx, method):
    import torch
    m, n, k = 333, 290, 610
    A = synth.matrix("scaled", k, m, k, 11, 6)
    B = synth.matrix("uniform", k, n, k + 3, 12)
    C = synth.matrix("uniform", m, n, m, 13)
    dA, dB = _dev(A, B)
    dC = torch.from_numpy(C).cuda()
    info = gbdgemm.GbdEmuInfo()
    rc = gbdgemm.gbd_ctx_dgemm(ctx, method, "T", "N", m, n, k, 1.25, dA, k, dB, k + 3, -0.5, dC, m, 0.0, info)
    assert rc == 0, gbdgemm.gbd_last_error()
    assert gbdgemm.gbd_sync_error(ctx) == 0
    ref = _direct(method, "T", "N", m, n, k, 1.25, dA, k, dB, k + 3, -0.5, C, m)
    assert np.array_equal(dC.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    assert info.path == {0: gbdgemm.GBD_PATH_NATIVE, 1: gbdgemm.GBD_PATH_SPLIT, 2: gbdgemm.GBD_PATH_MODULAR}[method]


def _halves(m, n, k, d, seed):
    return (synth.halves_matrix(m, k, m, seed, d, small_cols_from=k // 2),
            synth.halves_matrix(k, n, k, seed + 1, d, small_rows_below=k // 2))


def test_automatic_method_takes_the_fastest_certified_path(ctx, oracle_mod):
    import torch
    m = n = 96
    k = 1024
    seen = set()
    for d in (0, 18, 30):  # uniform data; a structure beyond 16 moduli but not 9 slices (when found); beyond both
        A, B = (synth.matrix("uniform", m, k, m, 40), synth.matrix("uniform", k, n, k, 41)) if d == 0 else \
            _halves(m, n, k, d, 40 + d)
        c = oracle_mod.certify("N", "N", m, n, k, A, m, B, k)
        want = (gbdgemm.GBD_PATH_MODULAR if c["moduli"] else
                gbdgemm.GBD_PATH_SPLIT if c["s"] <= 9 else gbdgemm.GBD_PATH_NATIVE)
        dA, dB = _dev(A, B)
        dC = torch.zeros(m * n, dtype=torch.float64, device="cuda")
        info = gbdgemm.GbdEmuInfo()
        rc = gbdgemm.gbd_ctx_dgemm(ctx, gbdgemm.GBD_METHOD_AUTO, "N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m,
                                   0.0, info)
        assert rc == 0, gbdgemm.gbd_last_error()
        assert gbdgemm.gbd_sync_error(ctx) == 0
        if want != gbdgemm.GBD_PATH_SPLIT or c["t"] == 63:  # the device may need one step more than the rule
            assert info.path == want or (want == gbdgemm.GBD_PATH_MODULAR and info.path == gbdgemm.GBD_PATH_SPLIT), \
                (d, c, info.path)
        seen.add(info.path)
        ref = oracle_mod.dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m)
        G = oracle_mod.abs_bound_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m)
        assert first_mismatch(dC.cpu().numpy(), ref, 2 * k * U * G, m) is None
    assert gbdgemm.GBD_PATH_MODULAR in seen and gbdgemm.GBD_PATH_NATIVE in seen


def test_pool_grows_per_stream(ctx):
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    A = torch.rand(512 * 512, dtype=torch.float64, device="cuda")
    C = torch.zeros(512 * 512, dtype=torch.float64, device="cuda")
    assert gbdgemm.gbd_ctx_pool_bytes(ctx) == 0
    assert gbdgemm.gbd_ctx_dgemm(ctx, gbdgemm.GBD_METHOD_MODULAR, "N", "N", 128, 128, 128, 1.0, A, 128, A, 128, 0.0,
                                 C, 128, stream=s1) == 0
    small = gbdgemm.gbd_ctx_pool_bytes(ctx)
    assert small >= gbdgemm.gbd_workspace_size(None, gbdgemm.GBD_METHOD_MODULAR, 128, 128, 128)[1]
    assert gbdgemm.gbd_ctx_dgemm(ctx, gbdgemm.GBD_METHOD_MODULAR, "N", "N", 512, 512, 512, 1.0, A, 512, A, 512, 0.0,
                                 C, 512, stream=s1) == 0
    grown = gbdgemm.gbd_ctx_pool_bytes(ctx)
    assert grown >= gbdgemm.gbd_workspace_size(None, gbdgemm.GBD_METHOD_MODULAR, 512, 512, 512)[1] > small
    assert gbdgemm.gbd_ctx_dgemm(ctx, gbdgemm.GBD_METHOD_SPLIT, "N", "N", 128, 128, 128, 1.0, A, 128, A, 128, 0.0,
                                 C, 128, stream=s2) == 0
    assert gbdgemm.gbd_ctx_pool_bytes(ctx) > grown  # a second stream gets its own block
    assert gbdgemm.gbd_sync_error(ctx, s1) == 0 and gbdgemm.gbd_sync_error(ctx, s2) == 0


def test_sync_error_reports_the_watchdog(ctx):
    assert gbdgemm.gbd_watchdog_selftest(20) == 0
    assert gbdgemm.gbd_sync_error(ctx) == gbdgemm.GBD_ERR_TIMEOUT
    assert gbdgemm.gbd_sync_error(ctx) == 0  # read and cleared


def test_context_grouped_call(ctx):
    import torch
    rng = np.random.default_rng(3)
    probs, hosts = [], []
    for q in range(6):
        m, n, k = (int(x) for x in rng.integers(40, 300, 3))
        A = synth.matrix("uniform", m, k, m, 100 + q)
        B = synth.matrix("uniform", k, n, k, 200 + q)
        dA, dB = _dev(A, B)
        dC = torch.zeros(m * n, dtype=torch.float64, device="cuda")
        hosts.append((m, n, k, dA, dB, dC))
        probs.append(dict(transa=b"N", transb=b"N", mode=q % 2, slices=0, m=m, n=n, k=k, alpha=1.0, beta=0.0, A=dA,
                          lda=m, B=dB, ldb=k, C=dC, ldc=m, tol=0.0))
    used = (ctypes.c_int * len(probs))()
    assert gbdgemm.gbd_ctx_dgemm_grouped(ctx, probs, used) == 0, gbdgemm.gbd_last_error()
    assert gbdgemm.gbd_sync_error(ctx) == 0
    for q, (m, n, k, dA, dB, dC) in enumerate(hosts):
        ref = torch.zeros(m * n, dtype=torch.float64, device="cuda")
        if q % 2 == 0:
            gbdgemm.check(gbdgemm.gbd_dgemm("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, ref, m))
        else:
            wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, used[q])
            ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
            gbdgemm.check(gbdgemm.gbd_dgemm_emu("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, ref, m, used[q], 0.0, ws,
                                                wsb))
        torch.cuda.synchronize()
        assert torch.equal(dC, ref)
