"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/gbdgemm.h declares; host-side argument checks answer without a GPU."""
from __future__ import annotations

import ctypes

import pytest

from paper_1609_00076_gb300 import build, gbdgemm


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gbdgemm.load()


def test_exports_every_declared_symbol(lib):
    names = gbdgemm.header_functions()
    assert "gbd_dgemm" in names
    raw = ctypes.CDLL(gbdgemm.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_version(lib):
    assert gbdgemm.gbd_version() >= 100


@pytest.mark.parametrize("args,code", [
    (("X", "N", 2, 2, 2, 2, 2, 2), 1), (("N", "Q", 2, 2, 2, 2, 2, 2), 2),
    (("N", "N", -1, 2, 2, 2, 2, 2), 3), (("N", "N", 2, -1, 2, 2, 2, 2), 4),
    (("N", "N", 2, 2, -1, 2, 2, 2), 5), (("N", "N", 3, 2, 2, 2, 2, 3), 8),
    (("T", "N", 2, 2, 3, 2, 3, 2), 8), (("N", "N", 2, 2, 3, 2, 2, 2), 10),
    (("N", "T", 2, 3, 2, 2, 2, 2), 10), (("N", "N", 3, 2, 2, 3, 2, 2), 13),
])
def test_argument_codes_without_gpu(lib, args, code):
    ta, tb, m, n, k, lda, ldb, ldc = args
    rc = gbdgemm.gbd_dgemm(ta, tb, m, n, k, 1.0, 0, lda, 0, ldb, 0.0, 0, ldc, stream=0)
    assert rc == code
    assert f"parameter {code}" in gbdgemm.gbd_last_error()


def test_empty_problem_is_a_no_op(lib):
    # m == 0 or n == 0 returns before any device work
    assert gbdgemm.gbd_dgemm("N", "N", 0, 5, 5, 1.0, 0, 1, 0, 5, 0.0, 0, 1, stream=0) == 0
    assert gbdgemm.gbd_dgemm("T", "T", 5, 0, 5, 1.0, 0, 5, 0, 1, 0.0, 0, 5, stream=0) == 0


def test_problem_struct_layout(lib):
    # the C side asserts the same size and offsets (grouped.cu)
    import ctypes
    P = gbdgemm.GbdProblem
    assert ctypes.sizeof(P) == 112
    assert P.m.offset == 16 and P.A.offset == 56 and P.tol.offset == 104
    assert P.ksplit.offset == 2 and P.mode.offset == 4  # ksplit sits in what was padding


def test_grouped_argument_errors_without_gpu(lib):
    bad = [dict(transa="N", transb="N", mode=0, m=4, n=4, k=4, alpha=1.0, beta=0.0, A=0, lda=2, B=0, ldb=4,
                C=0, ldc=4)]
    ws = gbdgemm.gbd_dgemm_grouped_workspace_size(bad)
    assert ws >= 256
    rc, plan = gbdgemm.gbd_grouped_plan_create(bad, 0, ws, stream=0)
    assert rc == gbdgemm.GBD_ERR_ARG
    assert "problem 0: parameter 8" in gbdgemm.gbd_last_error()
    bad[0]["lda"] = 4
    bad[0]["mode"] = 7
    rc, _ = gbdgemm.gbd_grouped_plan_create(bad, 0, ws, stream=0)
    assert rc == gbdgemm.GBD_ERR_ARG and "mode 7" in gbdgemm.gbd_last_error()
    bad[0]["mode"] = 0
    bad[0]["ksplit"] = 17
    rc, _ = gbdgemm.gbd_grouped_plan_create(bad, 0, ws, stream=0)
    assert rc == gbdgemm.GBD_ERR_ARG and "ksplit 17" in gbdgemm.gbd_last_error()


def test_ksplit_workspace_is_host_only(lib):
    # split-k native problems need part slots (one tile of doubles per part) and tile counters
    base = dict(transa="N", transb="N", mode=0, m=40, n=40, k=4096, alpha=1.0, beta=0.0, A=0, lda=40, B=0,
                ldb=4096, C=0, ldc=40, tile=32)
    w1 = gbdgemm.gbd_dgemm_grouped_workspace_size([dict(base, ksplit=1)])
    w8 = gbdgemm.gbd_dgemm_grouped_workspace_size([dict(base, ksplit=8)])
    assert w8 >= w1 + 4 * 8 * 32 * 32 * 8  # 2 x 2 tiles of 32, 8 parts each
    # a split beyond the 16-deep k-blocks is capped: k = 32 has two
    w16 = gbdgemm.gbd_dgemm_grouped_workspace_size([dict(base, k=32, ldb=32, ksplit=16)])
    w2 = gbdgemm.gbd_dgemm_grouped_workspace_size([dict(base, k=32, ldb=32, ksplit=2)])
    assert w16 == w2


def test_emu_workspace_size_is_host_only(lib):
    small = gbdgemm.gbd_dgemm_emu_workspace_size(100, 200, 300, 3)
    big = gbdgemm.gbd_dgemm_emu_workspace_size(100, 200, 300, 0)
    assert 0 < small < big
    assert gbdgemm.gbd_dgemm_emu_workspace_size(-1, 2, 3, 1) == 0


def test_emu_host_buffer_size_and_argument_codes_without_gpu(lib):
    import numpy as np
    ws = gbdgemm.gbd_dgemm_emu_workspace_size(100, 200, 300, 3)
    size = gbdgemm.gbd_dgemm_emu_host_buffer_size("T", "N", 100, 200, 300, 3)
    # packed A (300 x 100), B (300 x 200) and C (100 x 200), each 256-byte aligned, then the workspace
    assert size >= ws + 8 * (300 * 100 + 300 * 200 + 100 * 200)
    assert size <= ws + 8 * (300 * 100 + 300 * 200 + 100 * 200) + 4 * 256
    assert gbdgemm.gbd_dgemm_emu_host_buffer_size("N", "N", -1, 2, 3, 1) == 0
    a = np.zeros(4)
    # argument checks come before any device work
    assert gbdgemm.gbd_dgemm_emu_host("X", "N", 2, 2, 2, 1.0, a, 2, a, 2, 0.0, a, 2, 0, 0.0, None, 0, stream=0) == 1
    assert gbdgemm.gbd_dgemm_emu_host("N", "N", 2, 2, 2, 1.0, a, 1, a, 2, 0.0, a, 2, 0, 0.0, None, 0, stream=0) == 8
    assert gbdgemm.gbd_dgemm_emu_host("N", "N", 2, 2, 2, 1.0, a, 2, a, 2, 0.0, a, 1, 0, 0.0, None, 0, stream=0) == 13
    assert gbdgemm.gbd_dgemm_emu_host("N", "N", 0, 2, 2, 1.0, a, 1, a, 2, 0.0, a, 1, 0, 0.0, None, 0, stream=0) == 0
    assert gbdgemm.gbd_dgemm_emu_host("N", "N", 2, 2, 2, 1.0, a, 2, a, 2, 0.0, a, 2, 12, 0.0, None, 0, stream=0) == \
        gbdgemm.GBD_ERR_ARG


def test_request_stream_is_seeded_and_poisson():
    from paper_1609_00076_gb300 import serving
    a = serving.request_stream(3, 2000, rate=500.0)
    b = serving.request_stream(3, 2000, rate=500.0)
    assert [(r.arrival, r.m, r.n, r.k, r.mode) for r in a] == [(r.arrival, r.m, r.n, r.k, r.mode) for r in b]
    gaps = [y.arrival - x.arrival for x, y in zip(a, a[1:])]
    assert abs(sum(gaps) / len(gaps) - 1 / 500.0) < 0.1 / 500.0          # mean gap of a Poisson process
    big = sum(r.m == 4096 for r in a) / len(a)
    emu = sum(r.mode == serving.EMULATED for r in a) / len(a)
    assert 0.07 < big < 0.13 and 0.45 < emu < 0.55
    assert all(32 <= r.m <= 4096 and 32 <= r.k <= 4096 for r in a)


def test_emu_mod_moduli_are_coprime_minimal_and_enough(lib):
    import math
    all16 = gbdgemm.gbd_dgemm_emu_mod_moduli(62, 1)  # 2 2^124 = 2^125 needs all of them
    assert len(all16) == 16 and 2 ** 125 < math.prod(all16) < 2 ** 126
    assert all(2 <= p <= 256 for p in all16)  # symmetric residues within 128: exact in BF16
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(all16) for b in all16[i + 1:])
    for k in (1, 2, 3, 1000, 8192, 65537, 2 ** 31 - 1):
        for t in range(1, 63):
            mods = gbdgemm.gbd_dgemm_emu_mod_moduli(t, k)
            need = 2 * k * 2 ** (2 * t)  # 2 max |A'B'| for |A'|, |B'| <= 2^t
            if not mods:
                assert math.prod(all16) <= need, (t, k)
                continue
            assert mods == all16[:len(mods)]
            assert math.prod(mods) > need and math.prod(mods[:-1]) <= need, (t, k)
    assert len(gbdgemm.gbd_dgemm_emu_mod_moduli(44, 8192)) == 13  # 2 8192 2^88 = 2^102
    assert gbdgemm.gbd_dgemm_emu_mod_moduli(0, 10) == [] and gbdgemm.gbd_dgemm_emu_mod_moduli(10, 0) == []


def test_emu_mod_workspace_and_argument_codes_without_gpu(lib):
    import numpy as np
    few = gbdgemm.gbd_dgemm_emu_mod_workspace_size(100, 200, 300, 10)
    auto = gbdgemm.gbd_dgemm_emu_mod_workspace_size(100, 200, 300, 0)
    n10 = len(gbdgemm.gbd_dgemm_emu_mod_moduli(10, 300))
    # residues of both sides (2 bytes, k padded to 8) and one byte per result element, per modulus
    assert few >= n10 * (2 * 304 * (100 + 200) + 100 * 200)
    assert few < auto and gbdgemm.gbd_dgemm_emu_mod_workspace_size(-1, 2, 3, 0) == 0
    a = np.zeros(4)
    call = gbdgemm.gbd_dgemm_emu_mod
    assert call("X", "N", 2, 2, 2, 1.0, a, 2, a, 2, 0.0, a, 2, 0, 0.0, None, 0, stream=0) == 1
    assert call("N", "N", 2, 2, 2, 1.0, a, 2, a, 1, 0.0, a, 2, 0, 0.0, None, 0, stream=0) == 10
    assert call("N", "N", 2, 2, 2, 1.0, a, 2, a, 2, 0.0, a, 2, 63, 0.0, None, 0, stream=0) == gbdgemm.GBD_ERR_ARG
    assert call("N", "N", 2, 2, 2, 1.0, a, 2, a, 2, 0.0, a, 2, -2, 0.0, None, 0, stream=0) == gbdgemm.GBD_ERR_ARG
    assert call("N", "N", 2, 0, 2, 1.0, a, 2, a, 2, 0.0, a, 2, 0, 0.0, None, 0, stream=0) == 0


def test_level3_workspace_sizes_and_codes_without_gpu(lib):
    import numpy as np
    nat, emu = gbdgemm.GBD_MODE_NATIVE, gbdgemm.GBD_MODE_EMULATED
    # every call holds level-3 scratch (the solve: its diagonal blocks' inverses), emulated ones also
    # GEMM workspace
    assert 0 < gbdgemm.gbd_dtrsm_workspace_size("L", 1000, 300, nat) < gbdgemm.gbd_dtrsm_workspace_size("L", 1000, 300, emu)
    # the top split of 1000 is 512 + 488: both triangles' coupling products fit
    for shape in ((300, 488, 512), (300, 512, 488)):
        assert gbdgemm.gbd_dtrsm_workspace_size("R", 300, 1000, emu) >= gbdgemm.gbd_dgemm_emu_workspace_size(*shape, 0)
    assert 0 < gbdgemm.gbd_dtrmm_workspace_size("L", 1000, 300, nat) < gbdgemm.gbd_dtrmm_workspace_size("L", 1000, 300, emu)
    assert gbdgemm.gbd_dsyrk_workspace_size(700, 300, nat) == 512 * 512 * 8
    # 700 x 300 products are all below 1e8 flops (native); at 4096 x 256 the coupling block is modular
    assert gbdgemm.gbd_dsyrk_workspace_size(700, 300, emu) == 512 * 512 * 8
    assert gbdgemm.gbd_dsyrk_workspace_size(4096, 256, emu) >= 512 * 512 * 8 + \
        gbdgemm.gbd_dgemm_emu_mod_workspace_size(2048, 2048, 256, 0)
    assert gbdgemm.gbd_dtrmm_workspace_size("X", 10, 10, nat) == 0
    a = np.zeros(16)
    s = dict(stream=0)
    assert gbdgemm.gbd_dsyrk("X", "N", 2, 2, 1.0, a, 2, 0.0, a, 2, nat, 0.0, None, 0, **s) == 1
    assert gbdgemm.gbd_dsyrk("L", "X", 2, 2, 1.0, a, 2, 0.0, a, 2, nat, 0.0, None, 0, **s) == 2
    assert gbdgemm.gbd_dsyrk("L", "N", -1, 2, 1.0, a, 2, 0.0, a, 2, nat, 0.0, None, 0, **s) == 3
    assert gbdgemm.gbd_dsyrk("L", "N", 2, -1, 1.0, a, 2, 0.0, a, 2, nat, 0.0, None, 0, **s) == 4
    assert gbdgemm.gbd_dsyrk("L", "T", 2, 3, 1.0, a, 2, 0.0, a, 2, nat, 0.0, None, 0, **s) == 7
    assert gbdgemm.gbd_dsyrk("L", "N", 3, 2, 1.0, a, 3, 0.0, a, 2, nat, 0.0, None, 0, **s) == 10
    assert gbdgemm.gbd_dsyrk("L", "N", 0, 2, 1.0, a, 1, 0.0, a, 1, nat, 0.0, None, 0, **s) == 0
    for f in (gbdgemm.gbd_dtrmm, gbdgemm.gbd_dtrsm):
        assert f("X", "L", "N", "N", 2, 2, 1.0, a, 2, a, 2, nat, 0.0, None, 0, **s) == 1
        assert f("L", "X", "N", "N", 2, 2, 1.0, a, 2, a, 2, nat, 0.0, None, 0, **s) == 2
        assert f("L", "L", "X", "N", 2, 2, 1.0, a, 2, a, 2, nat, 0.0, None, 0, **s) == 3
        assert f("L", "L", "N", "X", 2, 2, 1.0, a, 2, a, 2, nat, 0.0, None, 0, **s) == 4
        assert f("L", "L", "N", "N", -1, 2, 1.0, a, 2, a, 2, nat, 0.0, None, 0, **s) == 5
        assert f("L", "L", "N", "N", 2, -1, 1.0, a, 2, a, 2, nat, 0.0, None, 0, **s) == 6
        assert f("R", "L", "N", "N", 2, 3, 1.0, a, 2, a, 2, nat, 0.0, None, 0, **s) == 9
        assert f("L", "L", "N", "N", 3, 2, 1.0, a, 3, a, 2, nat, 0.0, None, 0, **s) == 11
        assert f("L", "L", "N", "N", 3, 0, 1.0, a, 3, a, 3, nat, 0.0, None, 0, **s) == 0
        assert f("L", "L", "N", "N", 2, 2, 1.0, a, 2, a, 2, 5, 0.0, None, 0, **s) == gbdgemm.GBD_ERR_ARG


def test_context_workspace_sizes_without_gpu(lib):
    # the context's sizes are the entry points' own, computed on the host (no context needed)
    m, n, k = 300, 200, 1000
    cases = {gbdgemm.GBD_METHOD_NATIVE: 0,
             gbdgemm.GBD_METHOD_SPLIT: gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, 0),
             gbdgemm.GBD_METHOD_MODULAR: gbdgemm.gbd_dgemm_emu_mod_workspace_size(m, n, k, 0)}
    cases[gbdgemm.GBD_METHOD_AUTO] = max(cases[gbdgemm.GBD_METHOD_SPLIT], cases[gbdgemm.GBD_METHOD_MODULAR])
    for method, want in cases.items():
        assert gbdgemm.gbd_workspace_size(None, method, m, n, k) == (0, want)
    assert gbdgemm.gbd_workspace_size(None, 7, m, n, k)[0] == gbdgemm.GBD_ERR_ARG
    assert gbdgemm.gbd_workspace_size(None, 1, -1, n, k)[0] == 3
    assert gbdgemm.gbd_workspace_size(None, 1, m, n, -1)[0] == 5


def test_context_calls_refuse_cleanly_without_a_context(lib):
    assert gbdgemm.gbd_ctx_dgemm(None, 0, "N", "N", 2, 2, 2, 1.0, 0, 2, 0, 2, 0.0, 0, 2, stream=0) == \
        gbdgemm.GBD_ERR_ARG
    assert gbdgemm.gbd_sync_error(None, stream=0) == gbdgemm.GBD_ERR_ARG
    assert gbdgemm.gbd_ctx_pool_bytes(None) == 0
    gbdgemm.gbd_destroy(None)  # a no-op


def test_context_creation_reports_a_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: creation is tested with the GPU tests")
    rc, ctx = gbdgemm.gbd_create(0)
    assert rc in (gbdgemm.GBD_ERR_CUDA, gbdgemm.GBD_ERR_DEVICE) and not ctx.value


def test_serving_memory_accounting_without_gpu(lib):
    # a request holds its stored operands, C and (emulated) the modular workspace, plus slack
    from paper_1609_00076_gb300 import serving
    nat = serving.Request(0, 0.0, 300, 200, 100, "T", "N", serving.NATIVE)
    assert serving.Server.bytes_needed(nat) == 8 * (100 * 300 + 100 * 200 + 300 * 200) + 1024
    emu = serving.Request(1, 0.0, 300, 200, 100, "N", "T", serving.EMULATED)
    ws = gbdgemm.gbd_dgemm_emu_mod_workspace_size(300, 200, 100, 0)
    assert ws > 0
    assert serving.Server.bytes_needed(emu) == 8 * (300 * 100 + 200 * 100 + 300 * 200) + ws + 1024
    # a 4096^3 emulated request, the stream's largest, fits the 40 GB budget many times over
    big = serving.Request(2, 0.0, 4096, 4096, 4096, "N", "N", serving.EMULATED)
    assert 40e9 / serving.Server.bytes_needed(big) > 10
