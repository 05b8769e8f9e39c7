"""Modular problems in grouped plans (GBD_MODE_MODULAR): planned on the device by every run.

Bars: every modular problem's result is bit-identical to the single call gbd_dgemm_emu_mod
with bits = -1 (automatic, on the device) or with its fixed bits; a problem whose target no
bit count within 16 moduli certifies gives gbd_dgemm's bits (its FP64 fallback tiles run);
native problems and quick returns are unaffected; results meet the FP64 bound of the Dot2
oracle on a sample; a plan captured in a CUDA graph and replayed on new data in the same
buffers re-certifies that data; and plan creation does not wait for the stream.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import gbdgemm, synth
from test_grouped_gpu import bits_equal, make_batch, to_device

pytestmark = pytest.mark.gpu

_MODES = {"native": gbdgemm.GBD_MODE_NATIVE, "emu": gbdgemm.GBD_MODE_EMULATED, "mod": gbdgemm.GBD_MODE_MODULAR}


def descriptors(probs, tol=0.0):
    return [dict(transa=p["ta"], transb=p["tb"], mode=_MODES[p["mode"]], slices=p["slices"],
                 tile=p.get("tile", 0), m=p["m"], n=p["n"], k=p["k"], alpha=p["alpha"], beta=p["beta"],
                 A=p["dA"], lda=p["lda"], B=p["dB"], ldb=p["ldb"], C=p["dC"], ldc=p["ldc"], tol=tol)
            for p in probs]


def run_grouped(probs, tol=0.0):
    import torch
    arr = gbdgemm.problem_array(descriptors(probs, tol))
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    used = (ctypes.c_int * len(probs))()
    rc = gbdgemm.gbd_dgemm_grouped(arr, ws, wsb, slices_used=used)
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    return [p["dC"].cpu().numpy() for p in probs], list(used)


def run_single(p, tol=0.0):
    """The problem through its single-problem entry point, on a fresh copy of C."""
    import torch
    dC = torch.from_numpy(p["C"]).cuda()
    if p["mode"] == "mod":
        bits = p["slices"] if p["slices"] > 0 else -1
        wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(p["m"], p["n"], p["k"], bits)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        rc = gbdgemm.gbd_dgemm_emu_mod(p["ta"], p["tb"], p["m"], p["n"], p["k"], p["alpha"], p["dA"], p["lda"],
                                       p["dB"], p["ldb"], p["beta"], dC, p["ldc"], bits, tol, ws, wsb)
    else:
        rc = gbdgemm.gbd_dgemm(p["ta"], p["tb"], p["m"], p["n"], p["k"], p["alpha"], p["dA"], p["lda"], p["dB"],
                               p["ldb"], p["beta"], dC, p["ldc"])
    assert rc == 0, gbdgemm.gbd_last_error()
    torch.cuda.synchronize()
    gbdgemm.gbd_check_device_error()  # an infeasible single call marks the word; the batch does not
    return dC.cpu().numpy()


def _native_of(p):
    q = dict(p)
    q["mode"] = "native"
    return run_single(q)


def test_modular_batch_matches_single_calls(oracle_mod):
    probs = make_batch(51, 24, 32, 700, modes=("mod",), slices=(0,), kinds=("uniform", "scaled"),
                       alpha_beta=(1.5, -0.5))
    probs[3]["slices"] = 30  # fixed bits
    probs[7]["slices"] = 44
    to_device(probs)
    outs, used = run_grouped(probs)
    for p, out, s in zip(probs, outs, used):
        assert s == 0
        assert bits_equal(out, run_single(p)), (p["m"], p["n"], p["k"], p["slices"])
    for p, out in list(zip(probs, outs))[:5]:
        if p["slices"]:
            continue
        m, n, k = p["m"], p["n"], p["k"]
        ref = oracle_mod.dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                    p["beta"], p["C"], p["ldc"])
        G = oracle_mod.abs_bound_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                      p["beta"], p["C"], p["ldc"])
        got = synth.view(out, m, n, p["ldc"]).flatten(order="F")
        assert first_mismatch(got, ref, 2 * k * U * G, m) is None


@pytest.mark.parametrize("kernel", ["default", "single", "tile128"])
def test_large_problems_on_cta_pairs_match_single_calls(oracle_mod, monkeypatch, kernel):
    # problems with m, n, k >= 256 run their (256 x 256 tile, modulus) units on CTA pairs, the
    # others on single SMs (GBD_EMU_KERNEL=single, or tile 128 in the problem: all on single SMs,
    # the tile field naming the kernel of one problem); ragged sizes, a problem with
    # fixed bits (fewer moduli than the launch's largest count: its later units are skipped), one
    # with a target no bit count certifies (its units are skipped, its FP64 fallback runs) and a
    # quick return among them
    if kernel == "single":
        monkeypatch.setenv("GBD_EMU_KERNEL", "single")
    probs = make_batch(61, 16, 160, 1400, modes=("mod",), slices=(0,), kinds=("uniform", "scaled"),
                       alpha_beta=(1.5, -0.5))
    if kernel == "tile128":
        for p in probs[::2]:
            p["tile"] = 128
    big = [i for i, p in enumerate(probs) if min(p["m"], p["n"], p["k"]) >= 256]
    assert len(big) >= 4 and len(big) < len(probs)
    probs[big[0]]["slices"] = 20  # fixed bits: few moduli
    _structured(probs[big[1]])    # no certified bit count: the FP64 fallback
    probs[big[2]]["alpha"] = 0.0  # a quick return: C := beta C
    to_device(probs)
    outs, used = run_grouped(probs)
    for i, (p, out) in enumerate(zip(probs, outs)):
        want = _native_of(p) if i == big[1] else run_single(p)
        assert bits_equal(out, want), (i, p["m"], p["n"], p["k"], p["slices"])
    for i in big[3:5]:
        p, out = probs[i], outs[i]
        m, n, k = p["m"], p["n"], p["k"]
        ref = oracle_mod.dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                    p["beta"], p["C"], p["ldc"], rows=list(range(8)))
        G = oracle_mod.abs_bound_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                      p["beta"], p["C"], p["ldc"], rows=list(range(8)))
        got = synth.view(out, m, n, p["ldc"])[:8].flatten(order="F")
        assert first_mismatch(got, ref, 2 * k * U * G, 8) is None


def _structured(p, d=30):
    """Make problem p's operands the half-scaled structure (op(A)'s second half of k, op(B)'s first)."""
    k = p["k"]
    A = p["A"].reshape(-1, p["lda"])  # storage columns
    B = p["B"].reshape(-1, p["ldb"])
    if p["ta"] == "N":
        A[k // 2:, :] *= 2.0 ** -d
    else:
        A[:, k // 2:] *= 2.0 ** -d
    if p["tb"] == "N":
        B[:, : k // 2] *= 2.0 ** -d
    else:
        B[: k // 2, :] *= 2.0 ** -d


def test_mixed_batch_with_uncertifiable_problem_and_quick_returns(oracle_mod):
    probs = make_batch(52, 18, 40, 500, modes=("mod", "native", "emu"), slices=(0,), alpha_beta=(1.0, 0.5))
    for p in probs:
        if p["mode"] == "emu":
            p["slices"] = 6
    target = next(i for i, p in enumerate(probs) if p["mode"] == "mod" and p["k"] >= 64)
    _structured(probs[target])
    qi = next(i for i, p in enumerate(probs) if p["mode"] == "mod" and i != target)
    probs[qi]["alpha"] = 0.0  # a modular quick return: C := beta C
    to_device(probs)
    outs, used = run_grouped(probs)
    for i, (p, out) in enumerate(zip(probs, outs)):
        if i == target:  # no certified bit count: the FP64 fallback's bits
            assert bits_equal(out, _native_of(p))
            m, n, k = p["m"], p["n"], p["k"]
            ref = oracle_mod.dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                        p["beta"], p["C"], p["ldc"])
            G = oracle_mod.abs_bound_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"],
                                          p["ldb"], p["beta"], p["C"], p["ldc"])
            assert first_mismatch(synth.view(out, m, n, p["ldc"]).flatten(order="F"), ref, 2 * k * U * G, m) is None
        elif p["mode"] == "emu":
            import torch
            dC = torch.from_numpy(p["C"]).cuda()
            wsb = gbdgemm.gbd_dgemm_emu_workspace_size(p["m"], p["n"], p["k"], 6)
            ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
            gbdgemm.check(gbdgemm.gbd_dgemm_emu(p["ta"], p["tb"], p["m"], p["n"], p["k"], p["alpha"], p["dA"],
                                                p["lda"], p["dB"], p["ldb"], p["beta"], dC, p["ldc"], 6, 0.0, ws, wsb))
            torch.cuda.synchronize()
            assert bits_equal(out, dC.cpu().numpy())
        else:
            assert bits_equal(out, run_single(p)), (i, p["mode"])


def test_graph_replay_recertifies_new_data(oracle_mod):
    import torch
    probs = make_batch(53, 10, 64, 400, modes=("mod",), slices=(0,))
    to_device(probs)
    arr = gbdgemm.problem_array(descriptors(probs))
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, stream=s)
    assert rc == 0, gbdgemm.gbd_last_error()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert gbdgemm.gbd_grouped_plan_run(plan, stream=s) == 0
    # new data in the same buffers: problem 0 becomes the uncertifiable structure, the rest new values
    for i, p in enumerate(probs):
        p["A"] = synth.matrix("uniform", *((p["k"], p["m"]) if p["ta"] == "T" else (p["m"], p["k"])), p["lda"],
                              900 + i, pad=0.0)
        p["B"] = synth.matrix("uniform", *((p["n"], p["k"]) if p["tb"] == "T" else (p["k"], p["n"])), p["ldb"],
                              950 + i, pad=0.0)
        if i == 0:
            _structured(p)
        p["dA"].copy_(torch.from_numpy(p["A"]))
        p["dB"].copy_(torch.from_numpy(p["B"]))
        p["dC"].copy_(torch.from_numpy(p["C"]))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert gbdgemm.gbd_check_device_error() == 0
    for i, p in enumerate(probs):
        out = p["dC"].cpu().numpy()
        ref = _native_of(p) if i == 0 else run_single(p)
        assert bits_equal(out, ref), i
    gbdgemm.gbd_grouped_plan_destroy(plan)


def test_plan_creation_does_not_wait_for_the_stream():
    import torch
    probs = make_batch(54, 6, 64, 256, modes=("mod", "native"), slices=(0,))
    to_device(probs)
    arr = gbdgemm.problem_array(descriptors(probs))
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    # a first plan sets up the library's page-locked staging (allocation is a set-up step)
    rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, stream=s)
    assert rc == 0, gbdgemm.gbd_last_error()
    s.synchronize()
    gbdgemm.gbd_grouped_plan_destroy(plan)
    big = 4096
    A = torch.rand(big * big, dtype=torch.float64, device="cuda")
    C = torch.zeros(big * big, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    done = torch.cuda.Event()
    gbdgemm.check(gbdgemm.gbd_dgemm("N", "N", big, big, big, 1.0, A, big, A, big, 0.0, C, big, stream=s))  # ~0.1 s
    done.record(s)
    t0 = time.perf_counter()
    rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, stream=s)
    dt = time.perf_counter() - t0
    busy = not done.query()
    assert rc == 0, gbdgemm.gbd_last_error()
    assert busy, f"plan creation returned after the stream's earlier work ({dt * 1e3:.1f} ms)"
    assert gbdgemm.gbd_grouped_plan_run(plan, stream=s) == 0
    s.synchronize()
    gbdgemm.gbd_grouped_plan_destroy(plan)
    assert gbdgemm.gbd_check_device_error() == 0
