"""Failure detection without a GPU fault: a bounded device wait that runs out.

Every wait in the kernels gives up after a time limit, sets the device error word
and lets the kernel finish.  gbd_watchdog_selftest makes one such wait run out on
purpose (a barrier nothing arrives at); the host must then read GBD_ERR_TIMEOUT,
the word must be cleared by the read, and the context must still compute correctly.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_is_reported():
    import time

    import torch
    assert gbdgemm.gbd_check_device_error() == 0
    t0 = time.perf_counter()
    assert gbdgemm.gbd_watchdog_selftest(50) == 0
    rc = gbdgemm.gbd_check_device_error()
    dt = time.perf_counter() - t0
    assert rc == gbdgemm.GBD_ERR_TIMEOUT
    assert "gave up" in gbdgemm.gbd_last_error()
    assert 0.04 < dt < 5.0
    assert gbdgemm.gbd_check_device_error() == 0  # cleared by the read
    # the context is intact: a DGEMM still gives exact results on integer inputs
    m = n = k = 64
    A = synth.small_ints(1, m * k)
    B = synth.small_ints(2, k * n)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros(m * n, dtype=torch.float64, device="cuda")
    gbdgemm.check(gbdgemm.gbd_dgemm("N", "N", m, n, k, 1.0, dA, m, dB, k, 0.0, dC, m))
    torch.cuda.synchronize()
    ref = (A.reshape(k, m).T.astype(np.int64) @ B.reshape(n, k).T.astype(np.int64)).astype(np.float64)
    assert np.array_equal(dC.cpu().numpy().reshape(n, m).T, ref)


def test_selftest_argument_check():
    assert gbdgemm.gbd_watchdog_selftest(0) == gbdgemm.GBD_ERR_ARG
