"""Continuous-batching request loop over the grouped DGEMM.

Requests (C := alpha*op(A)*op(B) + beta*C of mixed sizes, each tagged native
FP64 or emulated with a target relative error) arrive over time.  The loop:

1. queues arrivals in order;
2. admits queued requests while the operands, C and workspace they need fit an
   HBM budget, allocating their operands on the device (they stay resident until
   the request completes);
3. whenever one of `slots` streams is free, forms a batch from admitted requests
   (FIFO, up to `max_batch` problems or `max_batch_flops` of work) and runs it as
   one grouped plan on that stream, so batches overlap on the device;
4. polls the batches' completion events, frees finished requests' memory and
   records each request's latency from arrival to observed completion.

Emulated requests are modular problems of the grouped plan: their precision is
certified and planned on the device inside the batch, so forming and launching a
batch never waits for the GPU.

Every GEMM step runs in the CUDA library; this module only schedules.  A
request's result does not depend on the batch it lands in: the grouped kernels
compute every problem exactly as the single-problem calls do.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import gbdgemm, synth

NATIVE = gbdgemm.GBD_MODE_NATIVE
# emulated requests run as modular problems: certified and planned on the device, so that making a
# batch's plan never waits for the stream
EMULATED = gbdgemm.GBD_MODE_MODULAR


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the run
    m: int
    n: int
    k: int
    transa: str
    transb: str
    mode: int
    tol: float = 0.0
    alpha: float = 1.0
    beta: float = 0.0
    seed: int = 0
    # filled by the server
    A: object = None
    B: object = None
    C: object = None
    lda: int = 0
    ldb: int = 0
    ldc: int = 0
    need: int = 0
    admitted: float = math.nan
    launched: float = math.nan
    completed: float = math.nan
    slices: int = 0
    batch: int = -1

    @property
    def flops(self) -> float:
        return 2.0 * self.m * self.n * self.k

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


def request_stream(seed: int, count: int, rate: float, big_fraction: float = 0.1, big: int = 4096,
                   emulated_fraction: float = 0.5, tol: float = 1e-14, lo: int = 32, hi: int = 2048,
                   start: float = 0.0) -> list[Request]:
    """Poisson arrivals at `rate` per second (rate <= 0: all at `start`); sizes log-uniform on
    [lo, hi] per dimension, a `big_fraction` of square `big` problems; a coin decides native or
    emulated (target relative error `tol`)."""
    gaps = synth.exponential(seed, count, rate) if rate > 0 else np.zeros(count)
    times = start + np.cumsum(gaps) - (gaps[0] if count else 0.0)
    sizes = synth.log_uniform_sizes(seed + 1, count, lo, hi)
    is_big = synth.coin(seed + 2, count, big_fraction)
    is_emu = synth.coin(seed + 3, count, emulated_fraction)
    flips = synth.coin(seed + 4, 2 * count)
    reqs = []
    for i in range(count):
        m, n, k = (big, big, big) if is_big[i] else (int(x) for x in sizes[i])
        reqs.append(Request(rid=i, arrival=float(times[i]), m=m, n=n, k=k, transa="T" if flips[2 * i] else "N",
                            transb="T" if flips[2 * i + 1] else "N", mode=EMULATED if is_emu[i] else NATIVE,
                            tol=tol if is_emu[i] else 0.0, seed=seed * 100003 + i))
    return reqs


@dataclass
class Batch:
    bid: int
    reqs: list
    stream: object
    event: object
    plan: object
    ws: object
    arr: object


@dataclass
class Report:
    requests: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    throughput_tflops: float
    requests_per_s: float
    batches: int
    mean_batch: float
    max_resident_gb: float
    extra: dict = field(default_factory=dict)

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k in ("requests", "wall_s", "p50_ms", "p99_ms", "mean_ms",
                                           "throughput_tflops", "requests_per_s", "batches", "mean_batch",
                                           "max_resident_gb")}
        d.update(self.extra)
        return d


class Server:
    """The request loop.  `budget_bytes` bounds the device memory held by admitted requests
    (operands, C and their share of the grouped workspace)."""

    def __init__(self, budget_bytes: float = 40e9, slots: int = 3, max_batch: int = 64,
                 max_batch_flops: float = 2.0e11, tuner=None, device: str = "cuda", keep_results: bool = False):
        import torch
        self.torch = torch
        self.budget = float(budget_bytes)
        self.max_batch = max_batch
        self.max_batch_flops = max_batch_flops
        self.tuner = tuner
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.keep_results = keep_results
        gbdgemm.load()

    # --- memory accounting ---
    @staticmethod
    def bytes_needed(r: Request) -> int:
        ra, ca = (r.k, r.m) if r.transa == "T" else (r.m, r.k)
        rb, cb = (r.n, r.k) if r.transb == "T" else (r.k, r.n)
        b = 8 * (ra * ca + rb * cb + r.m * r.n)
        if r.mode == EMULATED:
            b += gbdgemm.gbd_dgemm_emu_mod_workspace_size(r.m, r.n, r.k, 0)
        return b + 1024

    def _admit(self, r: Request, now: float) -> None:
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed(r.seed)
        ra, ca = (r.k, r.m) if r.transa == "T" else (r.m, r.k)
        rb, cb = (r.n, r.k) if r.transb == "T" else (r.k, r.n)
        r.lda, r.ldb, r.ldc = max(1, ra), max(1, rb), max(1, r.m)
        r.A = torch.empty(ra * ca, dtype=torch.float64, device=self.device).uniform_(-1.0, 1.0, generator=g)
        r.B = torch.empty(rb * cb, dtype=torch.float64, device=self.device).uniform_(-1.0, 1.0, generator=g)
        r.C = torch.zeros(r.m * r.n, dtype=torch.float64, device=self.device)
        r.admitted = now

    def _launch(self, bid: int, reqs: list, stream, now: float) -> Batch:
        torch = self.torch
        desc = [dict(transa=r.transa, transb=r.transb, mode=r.mode, slices=0, tile=0, m=r.m, n=r.n, k=r.k,
                     alpha=r.alpha, beta=r.beta, A=r.A, lda=r.lda, B=r.B, ldb=r.ldb, C=r.C, ldc=r.ldc, tol=r.tol)
                for r in reqs]
        if self.tuner is not None:
            self.tuner.apply(desc)
        arr = gbdgemm.problem_array(desc)
        wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
        ws = torch.empty(max(256, wsb), dtype=torch.uint8, device=self.device)
        used = (ctypes.c_int * len(reqs))()
        # the operands were written on torch's current stream: order the batch after them
        stream.wait_stream(torch.cuda.current_stream(self.device))
        rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb, slices_used=used, stream=stream)
        gbdgemm.check(rc)
        gbdgemm.check(gbdgemm.gbd_grouped_plan_run(plan, stream=stream))
        ev = torch.cuda.Event()
        ev.record(stream)
        for r, s in zip(reqs, used):
            r.slices = int(s)
            r.launched = now
            r.batch = bid
        return Batch(bid, reqs, stream, ev, plan, ws, arr)

    def run(self, requests: list[Request]) -> Report:
        """Serves `requests` (arrival times in seconds after the start, in real time) and returns
        the latency report."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue: deque = deque()
        admitted: deque = deque()
        free = list(self.streams)
        inflight: list[Batch] = []
        resident = 0
        max_resident = 0
        nb = 0
        batch_sizes = []
        done = []
        t0 = time.perf_counter()
        while pending or queue or admitted or inflight:
            now = time.perf_counter() - t0
            # arrivals
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # completions
            still = []
            for b in inflight:
                if b.event.query():
                    t = time.perf_counter() - t0
                    gbdgemm.gbd_grouped_plan_destroy(b.plan)
                    for r in b.reqs:
                        r.completed = t
                        resident -= r.need
                        if not self.keep_results:
                            r.A = r.B = r.C = None
                        done.append(r)
                    free.append(b.stream)
                else:
                    still.append(b)
            inflight = still
            # admission against the HBM budget (FIFO)
            while queue and resident + self.bytes_needed(queue[0]) <= self.budget:
                r = queue.popleft()
                r.need = self.bytes_needed(r)
                self._admit(r, now)
                resident += r.need
                max_resident = max(max_resident, resident)
                admitted.append(r)
            if queue and not admitted and not inflight and resident == 0:
                r = queue[0]
                raise RuntimeError(f"request {r.rid} needs {self.bytes_needed(r)} bytes, above the budget")
            # batching onto free slots
            while free and admitted:
                batch, work = [], 0.0
                while admitted and len(batch) < self.max_batch and (not batch or work + admitted[0].flops <=
                                                                      self.max_batch_flops):
                    r = admitted.popleft()
                    batch.append(r)
                    work += r.flops
                inflight.append(self._launch(nb, batch, free.pop(), now))
                batch_sizes.append(len(batch))
                nb += 1
            if inflight and not (free and admitted):
                time.sleep(20e-6)  # wait for a completion or an arrival
            elif not inflight and not admitted and pending:
                time.sleep(max(0.0, min(1e-3, pending[0].arrival - (time.perf_counter() - t0))))
        self.torch.cuda.synchronize()
        assert gbdgemm.gbd_check_device_error() == 0, gbdgemm.gbd_last_error()
        lat = np.array(sorted(r.latency for r in done)) * 1e3
        wall = max(r.completed for r in done) - min(r.arrival for r in done) if done else 0.0
        flops = sum(r.flops for r in done)
        return Report(requests=len(done), wall_s=wall, p50_ms=float(np.percentile(lat, 50)) if len(lat) else 0.0,
                      p99_ms=float(np.percentile(lat, 99)) if len(lat) else 0.0,
                      mean_ms=float(lat.mean()) if len(lat) else 0.0,
                      throughput_tflops=flops / wall / 1e12 if wall > 0 else 0.0,
                      requests_per_s=len(done) / wall if wall > 0 else 0.0, batches=nb,
                      mean_batch=float(np.mean(batch_sizes)) if batch_sizes else 0.0,
                      max_resident_gb=max_resident / 1e9)


def serving_benchmark(count: int = 2000, fractions=(0.5, 0.8, 0.95), seed: int = 5000, budget_gb: float = 40.0,
                      slots: int = 3, saturate_count: int | None = None) -> dict:
    """Measures the saturated request rate (all requests at t = 0), then serves Poisson streams at
    the given fractions of it; returns p50/p99 latency and throughput per rate."""
    server = Server(budget_bytes=budget_gb * 1e9, slots=slots)
    sat_n = saturate_count or count
    # warm-up: kernels, allocator, tensor-map encoder
    server.run(request_stream(seed - 1, 16, 0.0, big_fraction=0.0))
    sat = server.run(request_stream(seed, sat_n, 0.0))
    out = {"saturated": sat.as_dict(), "rates": []}
    for i, f in enumerate(fractions):
        rate = f * sat.requests_per_s
        rep = server.run(request_stream(seed + 10 * (i + 1), count, rate))
        d = rep.as_dict()
        d.update({"fraction_of_saturation": f, "rate_per_s": rate})
        out["rates"].append(d)
    out["config"] = {"requests_per_rate": count, "saturation_requests": sat_n,
                     "mix": "90% m,n,k log-uniform [32,2048], 10% 4096^3; 50/50 native FP64 / emulated (modular, "
                     "certified on the device) with target 1e-14; random transposes", "budget_gb": budget_gb,
                     "slots": slots}
    return out


def main():
    ap = argparse.ArgumentParser(description="continuous-batching DGEMM serving benchmark")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--slots", type=int, default=3)
    args = ap.parse_args()
    print(json.dumps(serving_benchmark(count=args.requests, budget_gb=args.budget_gb, slots=args.slots)))


if __name__ == "__main__":
    main()
