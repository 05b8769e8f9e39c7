#!/usr/bin/env python
"""Benchmark of the GB300 DGEMM library: C := alpha*op(A)*op(B) + beta*C.

Metric: DGEMM TFLOP/s (useful flops 2mnk per call) of the emulated DGEMM at FP64
accuracy -- the modular emulation (Ozaki scheme II: residues modulo coprime moduli,
automatic integer bits for the componentwise FP64 bound) -- with the split emulation
(automatic slices for the same bound) and the native FP64-MMA path measured beside it on
the same inputs, on the large square workload m = n = k = 8192 (FP64 operands uniform on
[-1, 1), N,N, alpha = 1, beta = 0; every input is larger than L2, so no flush is needed
between timed calls).  The dominant kernel's roofline is the BF16 tensor peak (residue
or slice products x 2mnk); the native path's is the FP64 peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one emulated DGEMM call on device-resident inputs.  Timing: W untimed
warm-up steps, then K steps between CUDA events on the launching stream, with a
barrier and a device synchronisation on both sides; the max over ranks is taken.
Multi-GPU runs are independent replicas (each rank its own problem, no
collective on the data path): value = total useful flops of all ranks / max time.

Rank 0 prints one JSON line.  `--impl reference` times the CPU oracle instead
(a bounded sample of rows of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DGEMM TFLOP/s vs FP64 peak: native vs emulated at FP64 accuracy; p99 latency"
M = N = K = 8192


def workload_name():
    return (f"dgemm m=n=k={M}, transa=transb=N, lda=ldb=ldc={M}, alpha=1, beta=0, "
            f"A,B uniform[-1,1) FP64")


PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# dram bytes (read + write) of the product launch of one 8192^3 call (dram__bytes_read.sum +
# dram__bytes_write.sum, one ncu pass at full size; the modular entry is the mean of two launches,
# 15.00 + 1.10 and 16.03 + 1.10 GB), None until captured for the current kernels
TRAFFIC_PER_LAUNCH = {"native": None, "emu": 79.827e9, "mod": 16.62e9}


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args, backend: str | None = None):
    """Replicas: one process per GPU, joined only for the start/stop barrier and the
    max-over-ranks time (NCCL on GPUs, gloo when there are none)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def replica_value(world: int, flops_per_step: float, steps: int, max_ms: float) -> float:
    """Whole-job TFLOP/s: every rank's useful flops over the slowest rank's time."""
    return world * flops_per_step * steps / (max_ms / 1000.0) / 1e12


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value: float, device=None) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------
# CPU oracle legs (the reference arm and the cpu_baseline)
# ------------------------------------------------------------------------------
_HOST_INPUTS: dict = {}


def host_inputs(seed: int):
    """The workload's A and B as column-major host buffers (cached per seed)."""
    from paper_1609_00076_gb300 import synth
    if seed not in _HOST_INPUTS:
        _HOST_INPUTS[seed] = (synth.matrix("uniform", M, K, M, seed, pad=0.0),
                              synth.matrix("uniform", K, N, K, seed + 1, pad=0.0))
    return _HOST_INPUTS[seed]


# kernels of one modular call with the bits chosen on the device: statistics and FP8 magnitude
# planes in one pass, the row merge (which also moves the planes to each row's scale), the
# certification product, the plan, the BF16 retry's planes, product and plan (three launches that
# return at once when the FP8 plan is feasible), residues, column scales, the products and the
# reconstruction of C from their parked residues
MOD_LAUNCHES = 11
# host threads (each with its own stream and device buffer) of the end-to-end measurement
E2E_STREAMS = 2



def oracle_sample(target_s: float, seed: int = 2000, want_rows: bool = False):
    """Times the CPU oracle on rows of the workload; returns (TFLOP/s, seconds, rows, threads), and
    with want_rows also the sampled row indices and the oracle's values there (nrows x N, column-major)."""
    import numpy as np

    import oracle
    oracle.build()
    A, B = host_inputs(seed)
    threads = oracle.num_threads()
    # calibrate on a few rows, then size the sample to about target_s seconds
    rows = list(range(0, M, M // 4))[:max(1, min(4, threads // 4 or 1))]
    t0 = time.perf_counter()
    oracle.dgemm_rows("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, None, M, rows=rows, nthreads=threads)
    dt = time.perf_counter() - t0
    per_row = dt / len(rows)
    nrows = int(max(1, min(M, target_s / max(per_row, 1e-6))))
    rows = [int(r) for r in (np.arange(nrows) * (M // max(nrows, 1))) % M]
    t0 = time.perf_counter()
    ref = oracle.dgemm_rows("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, None, M, rows=rows, nthreads=threads)
    dt = time.perf_counter() - t0
    flops = 2.0 * len(rows) * N * K
    if want_rows:
        return flops / dt / 1e12, dt, len(rows), threads, rows, ref
    return flops / dt / 1e12, dt, len(rows), threads


def accuracy_report(results: dict, rows, ref, seed: int = 2000) -> dict:
    """Error of each path's result against the oracle on the sampled rows: the largest |C - C_oracle|
    and its largest ratio to the componentwise bound 2 k 2^-53 (|A||B|)_ij."""
    import numpy as np
    A, B = host_inputs(seed)
    Ar = np.abs(A.reshape(K, M).T[rows, :])        # sampled rows of |A| (row-major)
    G = Ar @ np.abs(B.reshape(N, K).T)              # (nrows x N) of |A||B|
    Rv = ref.reshape(N, len(rows)).T                # oracle values, (nrows x N)
    out = {"rows": len(rows), "bound": "2 k 2^-53 (|A||B|)_ij"}
    for name, C in results.items():
        Cv = C.reshape(N, M).T[rows, :]
        err = np.abs(Cv - Rv)
        out[name] = {"max_abs_err": float(err.max()), "max_err_over_bound": float((err / (2 * K * 2.0 ** -53 * G)).max())}
    return out


def run_reference(args, world, rank, pg):
    if rank != 0:
        return 0
    steps, warm = args.steps, args.warmup
    vals = []
    total_t = 0.0
    info = None
    for i in range(warm + steps):
        v, dt, nrows, threads = oracle_sample(target_s=max(2.0, 60.0 / (warm + steps)), seed=2000 + i % 2)
        info = (nrows, threads)
        if i >= warm:
            vals.append(v)
            total_t += dt
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1000.0 * total_t / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "path": "cpu oracle (Dot2 triple loop)", "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": info[1], "kind": "oracle",
                         "sample": f"{info[0]} rows x {N} columns of the {M}^3 product per step"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------
# GPU legs
# ------------------------------------------------------------------------------
def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_ours(args, world, rank, local, pg):
    import torch

    from paper_1609_00076_gb300 import gbdgemm
    gbdgemm.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    seed = 2000 + rank
    A_h, B_h = host_inputs(seed)
    A = torch.from_numpy(A_h).to(dev)
    B = torch.from_numpy(B_h).to(dev)
    C = torch.zeros(M * N, dtype=torch.float64, device=dev)
    # the split path's workspace, allocated before the headline's: the split slice kernel's DRAM traffic
    # depends on where its slices land (36-39 GB per launch as the process's first large allocation,
    # 88-114 GB inside memory the modular workspace used)
    split_wsb = gbdgemm.gbd_dgemm_emu_workspace_size(M, N, K, 0)
    split_ws = torch.empty(split_wsb, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    flops = 2.0 * M * N * K

    # ---- the headline: the modular emulation, integer bits chosen on the device for the FP64 bound ----
    # (bits = -1: no host round trip inside a call; the timed steps pass no info, so nothing synchronises)
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(M, N, K, -1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    info = gbdgemm.GbdEmuInfo()

    def mod_step(s, report=False):
        info.record_phases = 1 if report else 0
        gbdgemm.check(gbdgemm.gbd_dgemm_emu_mod("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, C, M, -1, 0.0, ws, wsb,
                                                info if report else None, stream=s))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            mod_step(stream)
    torch.cuda.synchronize()
    gbdgemm.check(gbdgemm.gbd_check_device_error(stream))

    sampler = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    sampler.start()
    ev = _events(args.steps + 1)
    ev[0].record(stream)
    for i in range(args.steps):
        mod_step(stream)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clocks = sampler.stop()
    total_ms = ev[0].elapsed_time(ev[-1])
    gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
    total_ms = max_over_ranks(pg, total_ms, dev)
    value = replica_value(world, flops, args.steps, total_ms)
    # phases and the device's choice, from three further calls that read them back (untimed above)
    gemm_ms, prep_ms, recon_ms = [], [], []
    for _ in range(3):
        mod_step(stream, report=True)
        gemm_ms.append(info.gemm_ms)
        prep_ms.append(info.prep_ms)
        recon_ms.append(info.recon_ms)
    moduli, bits, bound_est = info.products, info.digit_bits, info.bound
    results = {"modular": C.cpu().numpy()} if rank == 0 else {}  # for the accuracy report (untimed)

    # ---- the split emulation on the same inputs (automatic slices at the same bound) ----
    split = split_measure(dev, stream, A, B, C, split_ws, split_wsb, steps=max(3, min(args.steps, 10)),
                          warmup=max(3, args.warmup))
    if rank == 0:
        results["split"] = C.cpu().numpy()

    # ---- native path on the same inputs ----
    def native_step(s):
        gbdgemm.check(gbdgemm.gbd_dgemm("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, C, M, stream=s))

    nat_calls = 2
    with torch.cuda.stream(stream):
        native_step(stream)
        torch.cuda.synchronize()
        nev = _events(nat_calls + 1)
        nev[0].record(stream)
        for i in range(nat_calls):
            native_step(stream)
            nev[i + 1].record(stream)
    torch.cuda.synchronize()
    nat_ms = statistics.mean(nev[i].elapsed_time(nev[i + 1]) for i in range(nat_calls))
    nat_tflops = flops / (nat_ms / 1000.0) / 1e12
    if rank == 0:
        results["native"] = C.cpu().numpy()

    # ---- end to end through the host-buffer C-ABI call (pinned host memory), copies inside the region ----
    # Each step is one gbd_dgemm_emu_mod_host call: upload of A and B, the emulated product, download of C.
    # Serial: one call at a time.  Overlapped (the reported value): E2E_STREAMS host threads, each driving
    # its own stream and device buffer, so the calls' transfers run under the other calls' products (a
    # call's own chain, upload, products and download, is about twice the products alone).
    A_p = torch.from_numpy(A_h).pin_memory()
    B_p = torch.from_numpy(B_h).pin_memory()
    C_p = [torch.empty(M * N, dtype=torch.float64).pin_memory() for _ in range(E2E_STREAMS)]
    hsize = gbdgemm.gbd_dgemm_emu_mod_host_buffer_size("N", "N", M, N, K, -1)
    hbufs = [torch.empty(hsize, dtype=torch.uint8, device=dev) for _ in range(E2E_STREAMS)]
    hstreams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(E2E_STREAMS - 1)]
    # enough calls that the first upload and the last download, which nothing hides, weigh little
    e2e_steps = max(2 * E2E_STREAMS, min(args.steps, 18))

    def host_call(i):
        j = i % E2E_STREAMS
        gbdgemm.check(gbdgemm.gbd_dgemm_emu_mod_host("N", "N", M, N, K, 1.0, A_p, M, B_p, K, 0.0, C_p[j], M, -1,
                                                     0.0, hbufs[j], hsize, None, stream=hstreams[j]))

    for i in range(E2E_STREAMS):  # untimed warm-up of every buffer and stream (first use of the pinned memory)
        host_call(i)
    torch.cuda.synchronize()
    e2e_sampler = ClockSampler(local)
    e2e_sampler.start()
    # serial
    sev = _events(e2e_steps + 1)
    sev[0].record(stream)
    for i in range(e2e_steps):
        host_call(0)
        sev[i + 1].record(stream)
    torch.cuda.synchronize()
    serial_ms = max_over_ranks(pg, sev[0].elapsed_time(sev[-1]), dev)
    # overlapped: the other streams start after e0 on stream 0; e1 on stream 0 after every stream is done
    e0, e1 = _events(2)
    e0.record(hstreams[0])
    for hs in hstreams[1:]:
        hs.wait_event(e0)
    errors = []

    def driver(t):
        try:
            for i in range(t, e2e_steps, E2E_STREAMS):
                host_call(i)
        except Exception as exc:  # re-raised below, on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=driver, args=(t,)) for t in range(E2E_STREAMS)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    if errors:
        raise errors[0]
    for hs in hstreams[1:]:
        last = torch.cuda.Event(enable_timing=False)
        last.record(hs)
        hstreams[0].wait_event(last)
    e1.record(hstreams[0])
    torch.cuda.synchronize()
    e2e_clocks = e2e_sampler.stop()
    gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
    e2e_ms = max_over_ranks(pg, e0.elapsed_time(e1), dev)
    e2e_val = replica_value(world, flops, e2e_steps, e2e_ms)
    e2e_serial = replica_value(world, flops, e2e_steps, serial_ms)
    del hbufs

    # ---- latency of small calls (256^3, the latency configuration) ----
    lat = small_call_latency(dev, stream)
    # ---- the FP64 tensor-core rate of this GPU (the native path's roofline), measured ----
    rc_probe, fp64_peak = gbdgemm.gbd_fp64_mma_probe(2000, stream=stream)  # about 0.3 s
    gbdgemm.check(rc_probe)
    # ---- the 8192^3 workload with wider exponent ranges (rank 0; the headline's inputs are overwritten) ----
    e_legs = exponent_legs(dev, stream, A, B, C, ws, wsb, split_ws, split_wsb) if rank == 0 else None
    del ws, split_ws
    # ---- grouped batch of 512 uneven problems, the serving loop, level-3 BLAS (rank 0, default size only) ----
    grouped = grouped_measure(dev, stream) if (rank == 0 and not args.no_extras) else None
    serving_rep = serving_measure() if (rank == 0 and not args.no_extras) else None
    level3 = level3_measure(dev, stream) if (rank == 0 and not args.no_extras) else None
    cpu_five = cpu_five_loop_measure() if (rank == 0 and not args.no_extras) else None

    if rank != 0:
        return 0
    peaks, src = load_peaks()
    # the modular call is about 10 ms, its timed region a fraction of a second: the burst peak applies
    bf16_burst = peaks["bf16_tflops"]
    bf16_sust = peaks.get("bf16_tflops_sustained", bf16_burst)
    g_ms = statistics.mean(gemm_ms)
    achieved = moduli * flops / (g_ms / 1000.0) / 1e12
    s_achieved = split["products"] * flops / (split["gemm_ms"] / 1000.0) / 1e12
    cpu_v, cpu_dt, cpu_rows, cpu_threads, rows, ref = oracle_sample(target_s=8.0, want_rows=True)
    accuracy = accuracy_report(results, rows, ref)
    launches_per_step = MOD_LAUNCHES
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(),
                   "path": "emulated at the FP64 bound: modular (Ozaki scheme II: residues modulo coprime moduli "
                           "<= 256 on tcgen05 BF16, Chinese remainder reconstruction; bits chosen on the device)",
                   "moduli": moduli, "integer_bits": bits, "certified_bound": bound_est,
                   "l2": f"inputs larger than L2 ({M * K * 8 >> 20} MiB each)", "parallelism": f"replicas x{world}"},
        "native": {"value": nat_tflops, "unit": "TFLOP/s", "ms_per_call": nat_ms, "frac_of_fp64_peak": nat_tflops / fp64_peak,
                   "fp64_peak": fp64_peak,
                   "fp64_peak_source": "measured: gbd_fp64_mma_probe (independent mma.sync.m16n8k16.f64 streams)"},
        "exponent_ranges": e_legs,
        "emulated_over_native": value / nat_tflops,
        "phases_ms": {"prep": statistics.mean(prep_ms), "products": g_ms, "reconstruction": statistics.mean(recon_ms)},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16_burst, "unit": "TFLOP/s",
                     "frac": achieved / bf16_burst, "frac_of_sustained": achieved / bf16_sust,
                     "traffic": TRAFFIC_PER_LAUNCH.get("mod"),
                     "kernel": "k_mod_gemm_pair (tcgen05 kind::f16 cta_group::2, BF16 -> FP32, residues parked; "
                               "(256 x 256 tile, modulus) work units, modulus-major)",
                     "peak_source": f"{src} bf16_tflops (burst: one call of about 10 ms)"},
        "split": {
            "value": split["value"], "unit": "TFLOP/s", "ms_per_call": split["ms"], "steps": split["steps"],
            "path": "emulated (split digits on tcgen05 BF16, FP64 bound)", "slices": split["slices"],
            "products": split["products"], "over_native": split["value"] / nat_tflops,
            "modular_over_split": value / split["value"],
            "phases_ms": {"prep": split["prep_ms"], "slice_gemm": split["gemm_ms"]},
            "roofline": {"bound": "tensor", "achieved": s_achieved, "peak": bf16_burst, "unit": "TFLOP/s",
                         "frac": s_achieved / bf16_burst, "traffic": TRAFFIC_PER_LAUNCH.get("emu"),
                         "kernel": "k_slice_gemm_pair (tcgen05 kind::f16 cta_group::2, BF16 -> FP32)",
                         "peak_source": f"{src} bf16_tflops (burst)"},
        },
        "latency": lat,
        "grouped": grouped,
        "serving": serving_rep,
        "level3": level3,
        "cpu_five_loop": cpu_five,
        "cpu_baseline": {"value": cpu_v, "unit": "TFLOP/s", "cores": cpu_threads, "kind": "oracle",
                         "sample": f"{cpu_rows} rows x {N} columns of the {M}^3 product ({cpu_dt:.1f} s)"},
        "accuracy": accuracy,
        "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": 2 * M * K * 8,
                "d2h_bytes_per_step": M * N * 8, "steps": e2e_steps,
                "call": f"gbd_dgemm_emu_mod_host (bits = -1), pinned host A, B, C; {E2E_STREAMS} host threads, one "
                        "stream and buffer each",
                "ms_per_step": e2e_ms / e2e_steps,
                "serial": {"value": e2e_serial, "ms_per_step": serial_ms / e2e_steps}, "clocks": e2e_clocks},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def split_measure(dev, stream, A, B, C, ws, wsb, steps: int, warmup: int):
    """Device time of gbd_dgemm_emu (the split emulation) on the headline inputs (automatic slices
    for the FP64 bound), and its phases, on the workspace `ws` of `wsb` bytes."""
    import torch

    from paper_1609_00076_gb300 import gbdgemm
    info = gbdgemm.GbdEmuInfo()

    def step(record):
        info.record_phases = 1 if record else 0
        gbdgemm.check(gbdgemm.gbd_dgemm_emu("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, C, M, 0, 0.0, ws, wsb,
                                            info, stream=stream))

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step(False)
    torch.cuda.synchronize()
    ev = _events(steps + 1)
    prep, prod = [], []
    ev[0].record(stream)
    for i in range(steps):
        step(True)
        prep.append(info.prep_ms)
        prod.append(info.gemm_ms)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
    ms = ev[0].elapsed_time(ev[-1]) / steps
    return {"ms": ms, "value": 2.0 * M * N * K / (ms / 1000.0) / 1e12, "slices": info.slices,
            "products": info.products, "prep_ms": statistics.mean(prep), "gemm_ms": statistics.mean(prod),
            "steps": steps}


def calls_only(dev, stream, which: str, steps: int, warmup: int, seed: int = 2000):
    """The headline's modular calls (bits chosen on the device) or the split calls (automatic
    slices) alone, on the headline's inputs at the current size: `warmup` calls, then `steps`
    calls timed with events (for profiling runs: nothing else launches)."""
    import torch

    from paper_1609_00076_gb300 import gbdgemm
    A_h, B_h = host_inputs(seed)
    A = torch.from_numpy(A_h).to(dev)
    B = torch.from_numpy(B_h).to(dev)
    C = torch.zeros(M * N, dtype=torch.float64, device=dev)
    if which == "split":
        wsb = gbdgemm.gbd_dgemm_emu_workspace_size(M, N, K, 0)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        res = split_measure(dev, stream, A, B, C, ws, wsb, steps=steps, warmup=warmup)
        res["path"] = "split"
        return res
    wsb = gbdgemm.gbd_dgemm_emu_mod_workspace_size(M, N, K, -1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)

    def call():
        gbdgemm.check(gbdgemm.gbd_dgemm_emu_mod("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, C, M, -1, 0.0, ws, wsb,
                                                None, stream=stream))

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            call()
    torch.cuda.synchronize()
    ev = _events(steps + 1)
    ev[0].record(stream)
    for i in range(steps):
        call()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
    ms = ev[0].elapsed_time(ev[-1]) / steps
    return {"path": "modular", "size": M, "ms": ms, "value": 2.0 * M * N * K / (ms / 1000.0) / 1e12,
            "steps": steps, "warmup": warmup}


def level3_measure(dev, stream, n: int = 8192, seed: int = 6000):
    """Device time of the GEMM-based DSYRK, DTRMM and DTRSM (side L, lower, N, non-unit) at n,
    native and emulated (each product at its FP64 bound): DSYRK on uniform[-1,1) A (the GEMM's
    inputs), the triangular operations on the well-conditioned A/n + 1.5 I; emulated DSYRK also
    on that diagonally dominant A ("dsyrk_dominant"): the off-diagonal entries of A A^T whose two
    small factors next to the 1.5 are themselves small need many more integer bits at the FP64
    bound (the row scale is set by the 1.5; more than 9 slices of the split emulation); the rows'
    small square sums keep the moduli that many bits need within 16."""
    import numpy as np
    import torch

    from paper_1609_00076_gb300 import gbdgemm, synth
    A = torch.from_numpy(synth.uniform_pm1(seed, n * n) / n).to(dev)
    A.view(n, n).diagonal().add_(1.5)
    Au = torch.from_numpy(synth.uniform_pm1(seed + 2, n * n)).to(dev)
    B0 = torch.from_numpy(synth.uniform_pm1(seed + 1, n * n)).to(dev)
    B = torch.empty_like(B0)
    C = torch.zeros(n * n, dtype=torch.float64, device=dev)
    out = {"n": n, "config": "dsyrk L,N n=k, A uniform[-1,1) (dsyrk_dominant: A/n + 1.5 I); dtrmm/dtrsm side L, "
                             "lower, N, non-unit, m=n, A/n + 1.5 I, B uniform[-1,1)",
           "flops": {"dsyrk": float(n) * n * n, "dtrmm": float(n) * n * n, "dtrsm": float(n) * n * n,
                     "dsyrk_dominant": float(n) * n * n}}
    for name, mode in (("native", gbdgemm.GBD_MODE_NATIVE), ("emulated", gbdgemm.GBD_MODE_EMULATED)):
        wsb = max(gbdgemm.gbd_dsyrk_workspace_size(n, n, mode), gbdgemm.gbd_dtrmm_workspace_size("L", n, n, mode),
                  gbdgemm.gbd_dtrsm_workspace_size("L", n, n, mode))
        ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
        calls = {
            "dsyrk": lambda: gbdgemm.gbd_dsyrk("L", "N", n, n, 1.0, Au, n, 0.0, C, n, mode, 0.0, ws, wsb, stream=stream),
            "dtrmm": lambda: gbdgemm.gbd_dtrmm("L", "L", "N", "N", n, n, 1.0, A, n, B, n, mode, 0.0, ws, wsb,
                                               stream=stream),
            "dtrsm": lambda: gbdgemm.gbd_dtrsm("L", "L", "N", "N", n, n, 1.0, A, n, B, n, mode, 0.0, ws, wsb,
                                               stream=stream),
        }
        if mode == gbdgemm.GBD_MODE_EMULATED:
            calls["dsyrk_dominant"] = lambda: gbdgemm.gbd_dsyrk("L", "N", n, n, 1.0, A, n, 0.0, C, n, mode, 0.0, ws, wsb,
                                                                stream=stream)
        res = {}
        for op, fn in calls.items():
            reps = 1 if mode == gbdgemm.GBD_MODE_NATIVE else 3
            with torch.cuda.stream(stream):
                B.copy_(B0)
                gbdgemm.check(fn())  # warm-up
                ev = _events(2 * reps)
                for r in range(reps):
                    B.copy_(B0)  # the triangular calls overwrite B: time each call alone
                    ev[2 * r].record(stream)
                    gbdgemm.check(fn())
                    ev[2 * r + 1].record(stream)
            torch.cuda.synchronize()
            ms = statistics.mean(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(reps))
            res[op] = {"ms": ms, "tflops": out["flops"][op] / (ms / 1000.0) / 1e12}
        gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
        out[name] = res
        del ws
    for op in ("dsyrk", "dtrmm", "dtrsm"):
        out[op + "_emulated_over_native"] = out["emulated"][op]["tflops"] / out["native"][op]["tflops"]
    return out


def exponent_legs(dev, stream, A, B, C, ws, wsb, split_ws, split_wsb, es=(8, 32), seed: int = 2100, calls: int = 3,
                  sample_rows: int = 16):
    """The 8192^3 workload with wider exponent ranges: entries uniform[-1,1) * 2^U, U uniform on {-e..e}.
    Each leg takes the fastest certified path (the modular emulation, else the split one, which
    computes natively when no slice count is certified), as gbd_ctx_dgemm's automatic method does;
    reports the path, its precision, the time per call and the error against the oracle on sampled
    rows.  A, B, C and the workspaces are reused (the headline's inputs are overwritten)."""
    import numpy as np
    import torch

    import oracle
    from paper_1609_00076_gb300 import gbdgemm, synth
    out = {}
    flops = 2.0 * M * N * K
    for e in es:
        g = torch.Generator(device=dev)
        g.manual_seed(seed + e)
        with torch.cuda.stream(stream):
            for X in (A, B):
                u = torch.empty(X.numel(), dtype=torch.float64, device=dev).uniform_(-1.0, 1.0, generator=g)
                ex = torch.randint(-e, e + 1, (X.numel(),), device=dev, generator=g, dtype=torch.int32)
                X.copy_(torch.ldexp(u, ex.to(torch.float64)))
                del u, ex
        stream.synchronize()
        info = gbdgemm.GbdEmuInfo()

        def call(report=False):
            info.record_phases = 0
            rc = gbdgemm.gbd_dgemm_emu_mod("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, C, M, 0, 0.0, ws, wsb,
                                           info if report else None, stream=stream)
            if rc == gbdgemm.GBD_ERR_LIMIT:  # no bit count within 16 moduli: the split emulation
                rc = gbdgemm.gbd_dgemm_emu("N", "N", M, N, K, 1.0, A, M, B, K, 0.0, C, M, 0, 0.0, split_ws, split_wsb,
                                           info if report else None, stream=stream)
            gbdgemm.check(rc)

        call(report=True)
        stream.synchronize()
        ev = _events(calls + 1)
        ev[0].record(stream)
        for i in range(calls):
            call()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[-1]) / calls
        gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
        path = {gbdgemm.GBD_PATH_MODULAR: "modular", gbdgemm.GBD_PATH_SPLIT: "split",
                gbdgemm.GBD_PATH_NATIVE: "native (no certified emulation)"}.get(info.path, str(info.path))
        leg = {"ms_per_call": ms, "tflops": flops / (ms / 1e3) / 1e12, "path": path}
        if info.path == gbdgemm.GBD_PATH_MODULAR:
            leg.update({"moduli": info.slices, "integer_bits": info.digit_bits, "certified_bound": info.bound})
        elif info.path == gbdgemm.GBD_PATH_SPLIT:
            leg.update({"slices": info.slices, "products": info.products, "certified_bound": info.bound})
        # the error against the oracle on sampled rows
        Ah, Bh, Ch = A.cpu().numpy(), B.cpu().numpy(), C.cpu().numpy()
        rows = sorted({int(r) for r in synth.splitmix64(seed + 7 * e, sample_rows) % M})
        ref = oracle.dgemm_rows("N", "N", M, N, K, 1.0, Ah, M, Bh, K, 0.0, None, M, rows=rows)
        G = oracle.abs_bound_rows("N", "N", M, N, K, 1.0, Ah, M, Bh, K, 0.0, None, M, rows=rows)
        got = Ch.reshape(N, M)[:, rows].flatten()
        err = np.abs(got - ref)
        leg["accuracy"] = {"rows": len(rows), "max_abs_err": float(err.max()),
                           "max_err_over_bound": float(np.max(err / (2 * K * 2.0 ** -53 * G)))}
        out[f"e{e}"] = leg
        del Ah, Bh, Ch
    return out


def grouped_batch(dev, count: int = 512, seed: int = 3000):
    """The grouped batch's problems (descriptors without a mode), the tensors they use and their
    flops: m, n, k each log-uniform on [32, 2048], random transposes, uniform[-1,1) operands."""
    import torch

    from paper_1609_00076_gb300 import synth
    sizes = synth.log_uniform_sizes(seed, count, 32, 2048)
    flips = synth.coin(seed + 1, 2 * count)
    keep, base = [], []
    for i in range(count):
        m, n, k = (int(x) for x in sizes[i])
        ta, tb = ("T" if flips[2 * i] else "N"), ("T" if flips[2 * i + 1] else "N")
        ra, ca = (k, m) if ta == "T" else (m, k)
        rb, cb = (n, k) if tb == "T" else (k, n)
        g = torch.Generator(device=dev)
        g.manual_seed(seed * 7919 + i)
        A = torch.empty(ra * ca, dtype=torch.float64, device=dev).uniform_(-1, 1, generator=g)
        B = torch.empty(rb * cb, dtype=torch.float64, device=dev).uniform_(-1, 1, generator=g)
        C = torch.zeros(m * n, dtype=torch.float64, device=dev)
        keep += [A, B, C]
        base.append(dict(transa=ta, transb=tb, m=m, n=n, k=k, alpha=1.0, beta=0.0, A=A, lda=ra, B=B, ldb=rb,
                         C=C, ldc=m, slices=0, tile=0, tol=0.0))
    flops = sum(2.0 * p["m"] * p["n"] * p["k"] for p in base)
    return base, keep, flops


def grouped_calls_only(dev, stream, which: str, count: int, steps: int, warmup: int):
    """One mode of the grouped batch alone (profiling runs): the plan of `count` problems in modular
    or split mode, `warmup` runs, then `steps` runs timed with events (nothing else launches)."""
    import torch

    from paper_1609_00076_gb300 import gbdgemm
    base, keep, flops = grouped_batch(dev, count)
    mode = gbdgemm.GBD_MODE_MODULAR if which == "grouped-modular" else gbdgemm.GBD_MODE_EMULATED
    arr = gbdgemm.problem_array([dict(p, mode=mode) for p in base])
    wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, stream=stream)
    gbdgemm.check(rc)
    try:
        for _ in range(warmup):
            gbdgemm.check(gbdgemm.gbd_grouped_plan_run(plan, stream=stream))
        torch.cuda.synchronize()
        ev = _events(steps + 1)
        ev[0].record(stream)
        for i in range(steps):
            gbdgemm.check(gbdgemm.gbd_grouped_plan_run(plan, stream=stream))
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
    finally:
        gbdgemm.gbd_grouped_plan_destroy(plan)
    ms = ev[0].elapsed_time(ev[-1]) / steps
    return {"path": which, "problems": count, "ms": ms, "tflops": flops / (ms / 1e3) / 1e12,
            "workspace_bytes": wsb, "steps": steps, "warmup": warmup}


def grouped_measure(dev, stream, count: int = 512, seed: int = 3000, reps: int = 3):
    """The grouped batch: 512 problems, m, n, k each log-uniform on [32, 2048], random transposes,
    uniform[-1,1).  Native problems take the autotuner's tile per output bucket and inner-dimension
    split per (output, k) bucket, split-emulated ones its kernel class per (output, k) bucket
    (measured here first; native also timed without the split); every plan
    run is captured once in a CUDA graph and replayed.  Modes: native FP64; modular (certified and
    planned on the device in every replay); split digits (slices certified when the plan is
    made).  TFLOP/s of graph replays (best of `reps`)."""
    import ctypes
    import tempfile

    import torch

    from paper_1609_00076_gb300 import autotune, gbdgemm
    base, keep, flops = grouped_batch(dev, count, seed)
    # the autotuner: native tile per output-size bucket, measured on this GPU into a fresh cache
    t0 = time.perf_counter()
    tuner = autotune.Autotuner(cache_path=os.path.join(tempfile.mkdtemp(), "tune.json"))
    tuner.tune_native_tiles(per_bucket=8, reps=2)
    tuner.tune_native_ksplit(per_bucket=32, reps=2)
    tuner.tune_emulated_class(per_bucket=8, reps=2)
    tune_s = time.perf_counter() - t0
    out = {"problems": count, "flops_per_batch": flops, "graph": True,
           "autotuner": {"seconds": tune_s, "native_tile_by_bucket": {b: e["tile"] for b, e in tuner.table.items()},
                         "native_ksplit_by_bucket": {b: e["ksplit"] for b, e in tuner.split_table.items()},
                         "emulated_class_by_bucket": {b: e["tile"] for b, e in tuner.emu_table.items()}}}
    for name, mode in (("native", gbdgemm.GBD_MODE_NATIVE), ("native_no_ksplit", gbdgemm.GBD_MODE_NATIVE),
                       ("emulated", gbdgemm.GBD_MODE_MODULAR), ("emulated_split", gbdgemm.GBD_MODE_EMULATED)):
        desc = [dict(p, mode=mode) for p in base]
        if name == "native_no_ksplit":
            for d in desc:
                d["ksplit"] = 1
        tuner.apply(desc)
        arr = gbdgemm.problem_array(desc)
        wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        used = (ctypes.c_int * count)()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, slices_used=used, stream=stream)
        gbdgemm.check(rc)
        create_ms = (time.perf_counter() - t0) * 1e3
        try:
            gbdgemm.check(gbdgemm.gbd_grouped_plan_run(plan, stream=stream))  # warm-up
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                gbdgemm.check(gbdgemm.gbd_grouped_plan_run(plan, stream=stream))
            with torch.cuda.stream(stream):
                graph.replay()
            torch.cuda.synchronize()  # the timed replays below must not overlap this one
            best = float("inf")
            for _ in range(reps):
                e0, e1 = _events(2)
                e0.record(stream)
                with torch.cuda.stream(stream):
                    graph.replay()
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            gbdgemm.check(gbdgemm.gbd_check_device_error(stream))
            del graph
        finally:
            gbdgemm.gbd_grouped_plan_destroy(plan)
        d = {"ms": best, "tflops": flops / (best / 1e3) / 1e12, "plan_create_ms": create_ms}
        if mode == gbdgemm.GBD_MODE_EMULATED:
            d["mean_slices"] = float(sum(max(0, u) for u in used) / count)
            d["fp64_fallbacks"] = int(sum(1 for u in used if u < 0))
        out[name] = d
        del ws
    out["emulated_over_native"] = out["emulated"]["tflops"] / out["native"]["tflops"]
    return out


def serving_measure(requests: int = 2000, seed: int = 5000):
    """The served request stream: the saturated rate of the mixed stream (all requests at once), then
    Poisson streams of `requests` requests at 0.5, 0.8 and 0.95 of it: p50/p99 latency and TFLOP/s
    per rate."""
    from paper_1609_00076_gb300 import serving
    return serving.serving_benchmark(count=requests, fractions=(0.5, 0.8, 0.95), seed=seed, budget_gb=40.0, slots=3,
                                     saturate_count=requests)


def cpu_five_loop_measure(n: int = 4096, seed: int = 7000, reps: int = 2):
    """The paper's own method on the host cores: the five-loop DGEMM (libgbdcpu.so) at n^3,
    N,N, alpha = 1, beta = 0, uniform[-1,1) inputs; wall time per call after one warm-up."""
    import numpy as np

    from paper_1609_00076_gb300 import cpu_blas, synth
    A = synth.matrix("uniform", n, n, n, seed, pad=0.0)
    B = synth.matrix("uniform", n, n, n, seed + 1, pad=0.0)
    C = np.zeros(n * n)
    assert cpu_blas.gbd_cpu_dgemm("N", "N", n, n, n, 1.0, A, n, B, n, 0.0, C, n) == 0  # warm-up
    t0 = time.perf_counter()
    for _ in range(reps):
        assert cpu_blas.gbd_cpu_dgemm("N", "N", n, n, n, 1.0, A, n, B, n, 0.0, C, n) == 0
    ms = (time.perf_counter() - t0) * 1000.0 / reps
    return {"value": 2.0 * n ** 3 / (ms / 1000.0) / 1e12, "unit": "TFLOP/s", "ms_per_call": ms,
            "threads": cpu_blas.max_threads(), "config": f"dgemm {n}^3 N,N alpha=1 beta=0, uniform[-1,1)",
            "blocking": cpu_blas.blocking(),
            "method": "GotoBLAS/BLIS five loops with packing, portable C micro-kernel, OpenMP over the packing "
                      "of op(B) and loop 3"}


def small_call_latency(dev, stream, calls: int = 200):
    """p50/p99 device latency of 256^3 native and emulated calls (one call per event pair)."""
    import torch

    from paper_1609_00076_gb300 import gbdgemm, synth
    m = n = k = 256
    A = torch.from_numpy(synth.matrix("uniform", m, k, m, 1, pad=0.0)).to(dev)
    B = torch.from_numpy(synth.matrix("uniform", k, n, k, 2, pad=0.0)).to(dev)
    C = torch.zeros(m * n, dtype=torch.float64, device=dev)
    slices = 7
    wsb = gbdgemm.gbd_dgemm_emu_workspace_size(m, n, k, slices)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    wsm_b = gbdgemm.gbd_dgemm_emu_mod_workspace_size(m, n, k, -1)
    wsm = torch.empty(wsm_b, dtype=torch.uint8, device=dev)
    out = {}
    for name, fn in (("native", lambda s: gbdgemm.gbd_dgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m, stream=s)),
                     ("emulated", lambda s: gbdgemm.gbd_dgemm_emu("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m,
                                                                 slices, 0.0, ws, wsb, None, stream=s)),
                     ("modular", lambda s: gbdgemm.gbd_dgemm_emu_mod("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m,
                                                                    -1, 0.0, wsm, wsm_b, None, stream=s))):
        with torch.cuda.stream(stream):
            for _ in range(5):
                gbdgemm.check(fn(stream))
            torch.cuda.synchronize()
            ev = _events(2 * calls)
            for i in range(calls):
                ev[2 * i].record(stream)
                gbdgemm.check(fn(stream))
                ev[2 * i + 1].record(stream)
            torch.cuda.synchronize()
        t = sorted(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(calls))
        out[name] = {"p50_ms": t[len(t) // 2], "p99_ms": t[min(len(t) - 1, int(0.99 * len(t)))]}
    out["config"] = ("256^3 N,N alpha=1 beta=0, uniform[-1,1); emulated with 7 slices; modular with its bits "
                     "chosen on the device; device time per call")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--only", choices=["grouped", "serving", "level3", "cpu", "modular", "split", "grouped-modular",
                                       "grouped-split"],
                    help="run only the grouped-batch, serving, level-3 or host five-loop measurement, only the "
                         "modular or split emulated calls at --size, or only one emulated mode of the grouped batch "
                         "of --problems problems (profiling runs), and print it")
    ap.add_argument("--problems", type=int, default=512, help="problems of the grouped batch in --only grouped-*")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the grouped-batch and serving measurements (profiling runs)")
    ap.add_argument("--size", type=int, default=8192,
                    help="m = n = k of the square workload (8192 is the benchmark; smaller sizes are for profiling)")
    args = ap.parse_args()
    global M, N, K
    M = N = K = args.size
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.only == "cpu":
        print(json.dumps(cpu_five_loop_measure()), flush=True)
        return 0
    if args.only:
        import torch

        from paper_1609_00076_gb300 import gbdgemm
        gbdgemm.load()
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        if args.only in ("modular", "split"):
            res = calls_only(dev, stream, args.only, args.steps, args.warmup)
        elif args.only == "grouped":
            res = grouped_measure(dev, stream, reps=1)
        elif args.only in ("grouped-modular", "grouped-split"):
            res = grouped_calls_only(dev, stream, args.only, args.problems, args.steps, args.warmup)
        elif args.only == "level3":
            res = level3_measure(dev, stream, n=args.size)
        else:
            res = serving_measure()
        print(json.dumps(res), flush=True)
        return 0
    world, rank, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank, pg)
        return run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
