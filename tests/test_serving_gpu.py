"""The continuous-batching request loop (paper_1609_00076_gb300.serving).

Checks: every request completes; each result is the same bits alone (single
native call, or the single modular call choosing its bits on the device from the
same target) as in the mix, for small requests and for 4096^3 ones (which the
single call runs on the CTA-pair kernels and the batch on the one-SM kernels);
results are within the bound of the oracle (sampled); the HBM budget is respected
while requests wait for admission.
"""
from __future__ import annotations

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import gbdgemm, serving

pytestmark = pytest.mark.gpu


def _alone(r):
    import torch
    dC = torch.zeros(r.m * r.n, dtype=torch.float64, device="cuda")
    if r.mode == serving.EMULATED:
        wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(r.m, r.n, r.k, -1)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        rc = gbdgemm.gbd_dgemm_emu_mod(r.transa, r.transb, r.m, r.n, r.k, r.alpha, r.A, r.lda, r.B, r.ldb, r.beta,
                                       dC, r.ldc, -1, r.tol, ws, wsb)
        assert rc == 0, gbdgemm.gbd_last_error()
    else:
        rc = gbdgemm.gbd_dgemm(r.transa, r.transb, r.m, r.n, r.k, r.alpha, r.A, r.lda, r.B, r.ldb, r.beta, dC, r.ldc)
        assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def test_mixed_stream_same_alone_and_in_the_mix(oracle_mod):
    reqs = serving.request_stream(7, 80, rate=2000.0, big_fraction=0.0, lo=32, hi=384)
    # and two 4096^3 requests among them, one of each kind
    for i, mode in enumerate((serving.NATIVE, serving.EMULATED)):
        reqs.append(serving.Request(rid=80 + i, arrival=reqs[20 + 10 * i].arrival, m=4096, n=4096, k=4096,
                                    transa="N", transb="T", mode=mode, tol=1e-14 if mode == serving.EMULATED else 0.0,
                                    seed=777 + i))
    srv = serving.Server(budget_bytes=4e9, slots=3, max_batch=16, keep_results=True)
    rep = srv.run(reqs)
    assert rep.requests == len(reqs)
    assert rep.p99_ms >= rep.p50_ms > 0
    assert rep.batches >= 2
    for r in reqs:
        mix = r.C.cpu().numpy()
        alone = _alone(r)
        assert np.array_equal(mix.view(np.uint64), alone.view(np.uint64)), (r.rid, r.mode, r.m, r.n, r.k)
    for r in reqs[:5]:
        A, B = r.A.cpu().numpy(), r.B.cpu().numpy()
        C0 = np.zeros(r.m * r.n)
        ref = oracle_mod.dgemm_rows(r.transa, r.transb, r.m, r.n, r.k, r.alpha, A, r.lda, B, r.ldb, r.beta, C0, r.ldc)
        G = oracle_mod.abs_bound_rows(r.transa, r.transb, r.m, r.n, r.k, r.alpha, A, r.lda, B, r.ldb, r.beta, C0,
                                      r.ldc)
        tol = 2 * r.k * U * G if r.mode == serving.NATIVE else np.maximum(2 * r.k * U, r.tol) * G
        assert first_mismatch(r.C.cpu().numpy(), ref, tol, r.m) is None


def test_admission_respects_budget():
    reqs = serving.request_stream(8, 40, rate=0.0, big_fraction=0.0, lo=256, hi=512, emulated_fraction=0.0)
    need = max(serving.Server.bytes_needed(r) for r in reqs)
    budget = 3.5 * need  # at most about three requests resident at a time
    srv = serving.Server(budget_bytes=budget, slots=2, max_batch=8)
    rep = srv.run(reqs)
    assert rep.requests == len(reqs)
    assert rep.max_resident_gb * 1e9 <= budget


def test_request_above_budget_is_refused():
    reqs = serving.request_stream(9, 2, rate=0.0, big_fraction=0.0, lo=512, hi=512)
    srv = serving.Server(budget_bytes=1e6, slots=1)
    with pytest.raises(RuntimeError):
        srv.run(reqs)
