"""Grouped calls (gbd_grouped_plan_* / gbd_dgemm_grouped): many uneven problems per launch.

Bars: every problem's result is bit-identical to the single-problem call with
the same arguments (native: gbd_dgemm; emulated: gbd_dgemm_emu with the same
slice count), i.e. the same alone and in any batch; emulated results are also
bit-identical to the CPU model of the method, native ones are within the FP64
bound of the Dot2 oracle (checked on a sample of problems); a plan replayed
from a CUDA graph gives the same bits again.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import gbdgemm, synth

pytestmark = pytest.mark.gpu


def make_batch(seed, count, lo, hi, modes=("native",), slices=(0,), kinds=("uniform",), alpha_beta=(1.0, 0.0)):
    """Host problems with log-uniform sizes, random transposes, padded leading dimensions."""
    sizes = synth.log_uniform_sizes(seed, count, lo, hi)
    flips = synth.coin(seed + 1, 2 * count)
    pick = synth.splitmix64(seed + 2, 3 * count)
    probs = []
    for i in range(count):
        m, n, k = (int(x) for x in sizes[i])
        ta = "T" if flips[2 * i] else "N"
        tb = "T" if flips[2 * i + 1] else "N"
        mode = modes[int(pick[3 * i] % len(modes))]
        s = slices[int(pick[3 * i + 1] % len(slices))]
        kind = kinds[int(pick[3 * i + 2] % len(kinds))]
        ra, ca = (k, m) if ta == "T" else (m, k)
        rb, cb = (n, k) if tb == "T" else (k, n)
        lda, ldb, ldc = ra + (i % 3), rb + (i % 2), m + 1
        A = synth.matrix(kind, ra, ca, lda, seed * 1000 + 3 * i, pad=0.0)
        B = synth.matrix(kind, rb, cb, ldb, seed * 1000 + 3 * i + 1, pad=0.0)
        C = synth.matrix("uniform", m, n, ldc, seed * 1000 + 3 * i + 2, pad=0.0)
        probs.append(dict(ta=ta, tb=tb, m=m, n=n, k=k, A=A, lda=lda, B=B, ldb=ldb, C=C, ldc=ldc,
                          mode=mode, slices=s, alpha=alpha_beta[0], beta=alpha_beta[1]))
    return probs


def to_device(probs):
    import torch
    for p in probs:
        p["dA"] = torch.from_numpy(p["A"]).cuda()
        p["dB"] = torch.from_numpy(p["B"]).cuda()
        p["dC"] = torch.from_numpy(p["C"]).cuda()
    torch.cuda.synchronize()


def descriptors(probs, tol=0.0):
    return [dict(transa=p["ta"], transb=p["tb"], mode=(gbdgemm.GBD_MODE_EMULATED if p["mode"] == "emu" else
                                                       gbdgemm.GBD_MODE_NATIVE),
                 slices=p["slices"], tile=p.get("tile", 0), m=p["m"], n=p["n"], k=p["k"], alpha=p["alpha"],
                 beta=p["beta"], A=p["dA"], lda=p["lda"], B=p["dB"], ldb=p["ldb"], C=p["dC"], ldc=p["ldc"], tol=tol)
            for p in probs]


def run_grouped(probs):
    import torch
    desc = descriptors(probs)
    arr = gbdgemm.problem_array(desc)
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    used = (ctypes.c_int * len(probs))()
    rc = gbdgemm.gbd_dgemm_grouped(arr, ws, wsb, slices_used=used)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    return [p["dC"].cpu().numpy() for p in probs], list(used)


def run_single(p, slices):
    """The same problem through the single-problem entry point, on a fresh copy of C."""
    import torch
    dC = torch.from_numpy(p["C"]).cuda()
    if p["mode"] == "emu":
        wsb = gbdgemm.gbd_dgemm_emu_workspace_size(p["m"], p["n"], p["k"], slices)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        rc = gbdgemm.gbd_dgemm_emu(p["ta"], p["tb"], p["m"], p["n"], p["k"], p["alpha"], p["dA"], p["lda"], p["dB"],
                                   p["ldb"], p["beta"], dC, p["ldc"], slices, 0.0, ws, wsb)
    else:
        rc = gbdgemm.gbd_dgemm(p["ta"], p["tb"], p["m"], p["n"], p["k"], p["alpha"], p["dA"], p["lda"], p["dB"],
                               p["ldb"], p["beta"], dC, p["ldc"])
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def bits_equal(a, b):
    return np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_native_batch_matches_single_calls(oracle_mod):
    probs = make_batch(11, 48, 32, 600, modes=("native",))
    to_device(probs)
    outs, _ = run_grouped(probs)
    for p, out in zip(probs, outs):
        assert bits_equal(out, run_single(p, 0)), (p["m"], p["n"], p["k"], p["ta"], p["tb"])
    for p, out in list(zip(probs, outs))[:6]:  # a sample against the oracle
        m, n, k = p["m"], p["n"], p["k"]
        ref = oracle_mod.dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                    p["beta"], p["C"], p["ldc"])
        G = oracle_mod.abs_bound_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                      p["beta"], p["C"], p["ldc"])
        got = synth.view(out, m, n, p["ldc"]).flatten(order="F")
        assert first_mismatch(got, ref, 2 * k * U * G, m) is None


@pytest.mark.parametrize("tile", [32, 64])
def test_native_tile_override_same_bits(tile):
    probs = make_batch(12, 12, 40, 300, modes=("native",))
    for p in probs:
        p["tile"] = tile
    to_device(probs)
    outs, _ = run_grouped(probs)
    for p, out in zip(probs, outs):
        assert bits_equal(out, run_single(p, 0))


def test_emulated_batch_matches_single_calls_and_model(oracle_mod):
    probs = make_batch(21, 16, 32, 400, modes=("emu",), slices=(3, 5, 7, 8), alpha_beta=(1.5, -0.5))
    to_device(probs)
    outs, used = run_grouped(probs)
    for p, out, s in zip(probs, outs, used):
        assert s == p["slices"]
        assert bits_equal(out, run_single(p, s))
        m, n, k = p["m"], p["n"], p["k"]
        ref = oracle_mod.ozaki_dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                          p["beta"], p["C"], p["ldc"], s)
        got = synth.view(out, m, n, p["ldc"]).flatten(order="F")
        assert first_mismatch(got, ref, None, m) is None


def test_emulated_two_kernel_classes(oracle_mod):
    # m, n >= 1024 with k >= 2048 go to the two-SM 256 x 256 kernel, the others to the one-SM kernel;
    # ragged sizes, transposes and several slice counts (one launch per kernel and slice count)
    probs = make_batch(23, 8, 120, 700, modes=("emu",), slices=(3, 5, 9), alpha_beta=(-0.75, 1.25))
    for i, (m, n, k, ta, tb, s) in enumerate([(1030, 1100, 2100, "N", "T", 3), (1100, 1030, 2049, "T", "N", 4)]):
        ra, ca = (k, m) if ta == "T" else (m, k)
        rb, cb = (n, k) if tb == "T" else (k, n)
        probs.append(dict(ta=ta, tb=tb, m=m, n=n, k=k, lda=ra + 1, ldb=rb, ldc=m + 1, mode="emu", slices=s,
                          alpha=-0.75, beta=1.25, A=synth.matrix("uniform", ra, ca, ra + 1, 7000 + i, pad=0.0),
                          B=synth.matrix("uniform", rb, cb, rb, 7100 + i, pad=0.0),
                          C=synth.matrix("uniform", m, n, m + 1, 7200 + i, pad=0.0)))
    to_device(probs)
    outs, used = run_grouped(probs)
    for p, out, s in zip(probs, outs, used):
        assert s == p["slices"]
        m, n, k = p["m"], p["n"], p["k"]
        ref = oracle_mod.ozaki_dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                          p["beta"], p["C"], p["ldc"], s)
        got = synth.view(out, m, n, p["ldc"]).flatten(order="F")
        assert first_mismatch(got, ref, None, m) is None, (m, n, k, s)
        assert bits_equal(out, run_single(p, s))


def test_emulated_automatic_slices_within_bound(oracle_mod):
    probs = make_batch(22, 10, 48, 500, modes=("emu",), slices=(0,), kinds=("uniform", "scaled"))
    to_device(probs)
    outs, used = run_grouped(probs)
    for p, out, s in zip(probs, outs, used):
        assert 1 <= s <= 9
        assert bits_equal(out, run_single(p, s))
        m, n, k = p["m"], p["n"], p["k"]
        ref = oracle_mod.dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                    p["beta"], p["C"], p["ldc"])
        G = oracle_mod.abs_bound_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                      p["beta"], p["C"], p["ldc"])
        got = synth.view(out, m, n, p["ldc"]).flatten(order="F")
        assert first_mismatch(got, ref, 2 * k * U * G, m) is None


def test_mixed_batch_with_quick_returns():
    probs = make_batch(31, 20, 32, 300, modes=("native", "emu"), slices=(4, 6))
    probs[0]["alpha"] = 0.0           # C := beta*C, A and B not read
    probs[1]["k"] = 0                 # C := beta*C
    probs[1]["beta"] = -2.0
    probs[2]["alpha"], probs[2]["beta"] = 0.0, 1.0   # nothing happens
    probs[3]["beta"] = 0.0
    probs[3]["C"][:] = np.nan         # beta == 0: C not read
    to_device(probs)
    outs, _ = run_grouped(probs)
    for p, out in zip(probs, outs):
        assert bits_equal(out, run_single(p, p["slices"]))
    p3 = probs[3]
    assert np.isfinite(synth.view(outs[3], p3["m"], p3["n"], p3["ldc"])).all()


def test_plan_replay_and_cuda_graph():
    import torch
    probs = make_batch(41, 24, 32, 256, modes=("native", "emu"), slices=(5,))
    to_device(probs)
    desc = descriptors(probs)
    arr = gbdgemm.problem_array(desc)
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, stream=s)
    assert rc == 0, gbdgemm.gbd_last_error()
    try:
        c0 = [p["dC"].clone() for p in probs]
        # plain run
        assert gbdgemm.gbd_grouped_plan_run(plan, stream=s) == 0
        torch.cuda.synchronize()
        first = [p["dC"].cpu().numpy() for p in probs]
        # capture the run in a CUDA graph and replay it on restored inputs
        for p, c in zip(probs, c0):
            p["dC"].copy_(c)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            rc = gbdgemm.gbd_grouped_plan_run(plan, stream=torch.cuda.current_stream())
        assert rc == 0, gbdgemm.gbd_last_error()
        for p, c in zip(probs, c0):
            p["dC"].copy_(c)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert gbdgemm.gbd_check_device_error() == 0
        replayed = [p["dC"].cpu().numpy() for p in probs]
        for a, b in zip(first, replayed):
            assert bits_equal(a, b)
        # the graph reads its inputs afresh: new A values give the single-call result for them
        probs[0]["dA"].mul_(2.0)
        probs[0]["A"] = probs[0]["dA"].cpu().numpy()
        for p, c in zip(probs, c0):
            p["dC"].copy_(c)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert bits_equal(probs[0]["dC"].cpu().numpy(), run_single(probs[0], probs[0]["slices"]))
    finally:
        gbdgemm.gbd_grouped_plan_destroy(plan)
