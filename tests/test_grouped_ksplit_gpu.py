"""Split inner dimension in the grouped FP64 kernel (gbd_problem.ksplit) and the tuner that picks it.

Bars: with ksplit parts per tile, every result is within the FP64 bound of the Dot2 oracle
(the parts' sums add k/S-deep partial sums, still a recursive sum over k); the bits do not
depend on the order the parts run in (two runs and a CUDA-graph replay agree bit for bit, and
the counters are ready for the next run); ksplit = 1 gives gbd_dgemm's bits; the tuner's
table, applied to a batch, keeps those properties; an emulated problem's kernel class (the
tile field: one-SM or two-SM) does not change its bits.
"""
from __future__ import annotations

import os
import tempfile

import numpy as np
import pytest

from conftest import U, first_mismatch
from paper_1609_00076_gb300 import autotune, gbdgemm, synth
from test_grouped_gpu import bits_equal, make_batch, to_device

pytestmark = pytest.mark.gpu


def _desc(probs, ksplit, tile=0):
    return [dict(transa=p["ta"], transb=p["tb"], mode=gbdgemm.GBD_MODE_NATIVE, ksplit=ksplit, tile=tile,
                 m=p["m"], n=p["n"], k=p["k"], alpha=p["alpha"], beta=p["beta"], A=p["dA"], lda=p["lda"],
                 B=p["dB"], ldb=p["ldb"], C=p["dC"], ldc=p["ldc"]) for p in probs]


def _reset(probs):
    import torch
    for p in probs:
        p["dC"].copy_(torch.from_numpy(p["C"]))
    torch.cuda.synchronize()


def _run(probs, desc, graph=False):
    """Runs the plan twice (directly, or created once and replayed from a graph twice); returns both
    results."""
    import torch
    arr = gbdgemm.problem_array(desc)
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, stream=s)
    assert rc == 0, gbdgemm.gbd_last_error()
    outs = []
    try:
        g = None
        if graph:
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                assert gbdgemm.gbd_grouped_plan_run(plan, stream=s) == 0
        for _ in range(2):
            _reset(probs)
            if g is not None:
                with torch.cuda.stream(s):
                    g.replay()
            else:
                assert gbdgemm.gbd_grouped_plan_run(plan, stream=s) == 0
            s.synchronize()
            assert gbdgemm.gbd_check_device_error() == 0
            outs.append([p["dC"].cpu().numpy() for p in probs])
    finally:
        gbdgemm.gbd_grouped_plan_destroy(plan)
    return outs


def _check_bound(oracle_mod, probs, outs):
    for p, out in zip(probs, outs):
        m, n, k = p["m"], p["n"], p["k"]
        ref = oracle_mod.dgemm_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                    p["beta"], p["C"], p["ldc"])
        G = oracle_mod.abs_bound_rows(p["ta"], p["tb"], m, n, k, p["alpha"], p["A"], p["lda"], p["B"], p["ldb"],
                                      p["beta"], p["C"], p["ldc"])
        got = synth.view(out, m, n, p["ldc"]).flatten(order="F")
        assert first_mismatch(got, ref, 2 * k * U * G, m) is None, (m, n, k)


@pytest.mark.parametrize("ksplit,tile,graph", [(2, 32, False), (4, 64, True), (16, 32, True), (16, 0, False)])
def test_split_k_within_bound_and_order_independent(oracle_mod, ksplit, tile, graph):
    # small outputs with a deep k (the case split-k serves), plus a few ordinary problems
    probs = make_batch(71, 10, 24, 100, alpha_beta=(1.25, -0.5))
    for i, p in enumerate(probs[:7]):  # deepen k: 700..3000, with odd values for ragged parts
        k = 700 + 331 * i
        ra, ca = (k, p["m"]) if p["ta"] == "T" else (p["m"], k)
        rb, cb = (p["n"], k) if p["tb"] == "T" else (k, p["n"])
        p["k"], p["lda"], p["ldb"] = k, ra + 1, rb
        p["A"] = synth.matrix("uniform", ra, ca, ra + 1, 7100 + i, pad=0.0)
        p["B"] = synth.matrix("uniform", rb, cb, rb, 7200 + i, pad=0.0)
    to_device(probs)
    outs = _run(probs, _desc(probs, ksplit, tile), graph=graph)
    for a, b in zip(outs[0], outs[1]):
        assert bits_equal(a, b)  # the parts' order of completion does not show in the bits
    _check_bound(oracle_mod, probs[:6], outs[0][:6])


def test_split_one_is_the_unsplit_kernel():
    import torch
    probs = make_batch(72, 8, 32, 300, alpha_beta=(0.75, 0.25))
    to_device(probs)
    o1 = _run(probs, _desc(probs, 1, 32))[0]
    o0 = _run(probs, _desc(probs, 0, 32))[0]
    for p, a, b in zip(probs, o0, o1):
        assert bits_equal(a, b)
        dC = torch.from_numpy(p["C"]).cuda()
        gbdgemm.check(gbdgemm.gbd_dgemm(p["ta"], p["tb"], p["m"], p["n"], p["k"], p["alpha"], p["dA"], p["lda"],
                                        p["dB"], p["ldb"], p["beta"], dC, p["ldc"]))
        torch.cuda.synchronize()
        # the single call's kernel tiles differ from the grouped 32 x 32 tile only in staging: same k order
        assert bits_equal(a, dC.cpu().numpy())


def test_tuner_chooses_a_split_and_the_batch_keeps_its_properties(oracle_mod):
    tuner = autotune.Autotuner(cache_path=os.path.join(tempfile.mkdtemp(), "tune.json"))
    table = tuner.tune_native_ksplit(out_buckets=range(5, 6), k_buckets=range(10, 12), per_bucket=8, reps=1)
    assert set(table) == {"5_10", "5_11"}
    for e in table.values():
        assert e["ksplit"] in autotune.KSPLITS and set(e["ms"]) == {str(s) for s in autotune.KSPLITS}
    reloaded = autotune.Autotuner(cache_path=tuner.cache_path)
    assert reloaded.split_table == table
    probs = make_batch(73, 6, 32, 63)
    for i, p in enumerate(probs):
        k = 1100 + 200 * i
        ra, ca = (k, p["m"]) if p["ta"] == "T" else (p["m"], k)
        rb, cb = (p["n"], k) if p["tb"] == "T" else (k, p["n"])
        p["k"], p["lda"], p["ldb"] = k, ra, rb
        p["A"] = synth.matrix("uniform", ra, ca, ra, 7300 + i, pad=0.0)
        p["B"] = synth.matrix("uniform", rb, cb, rb, 7400 + i, pad=0.0)
    to_device(probs)
    desc = tuner.apply(_desc(probs, 0))
    assert all(d["ksplit"] == tuner.ksplit_for(d["m"], d["n"], d["k"]) for d in desc)
    outs = _run(probs, desc)
    for a, b in zip(outs[0], outs[1]):
        assert bits_equal(a, b)
    _check_bound(oracle_mod, probs, outs[0])


def test_emulated_kernel_class_choice_keeps_the_bits():
    # the tile field of an emulated problem names its kernel (128: one-SM, 256: two-SM); both give
    # the single call's bits, and the tuner's choice per bucket is one of them
    import torch
    from test_grouped_gpu import run_single
    tuner = autotune.Autotuner(cache_path=os.path.join(tempfile.mkdtemp(), "tune.json"))
    table = tuner.tune_emulated_class(out_buckets=range(10, 11), k_buckets=range(10, 11), per_bucket=4, reps=1)
    assert set(table) == {"10_10"} and table["10_10"]["tile"] in autotune.EMU_CLASSES
    probs = make_batch(74, 4, 1024, 1500, modes=("emu",), slices=(6,), alpha_beta=(1.0, 0.5))
    to_device(probs)
    outs = {}
    for tile in (128, 256, 0):
        for p in probs:
            p["dC"].copy_(torch.from_numpy(p["C"]))
        desc = [dict(transa=p["ta"], transb=p["tb"], mode=gbdgemm.GBD_MODE_EMULATED, slices=6, tile=tile, m=p["m"],
                     n=p["n"], k=p["k"], alpha=p["alpha"], beta=p["beta"], A=p["dA"], lda=p["lda"], B=p["dB"],
                     ldb=p["ldb"], C=p["dC"], ldc=p["ldc"]) for p in probs]
        if tile == 0:
            tuner.apply(desc)
        arr = gbdgemm.problem_array(desc)
        wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        assert gbdgemm.gbd_dgemm_grouped(arr, ws, wsb) == 0, gbdgemm.gbd_last_error()
        torch.cuda.synchronize()
        outs[tile] = [p["dC"].cpu().numpy() for p in probs]
    for q, p in enumerate(probs):
        ref = run_single(p, 6)
        for tile in (128, 256, 0):
            assert bits_equal(outs[tile][q], ref), (tile, p["m"], p["n"], p["k"])
