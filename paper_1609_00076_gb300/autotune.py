"""Measured tile selection for grouped native problems, cached as JSON.

The grouped FP64-MMA kernel can run each problem with 32 x 32 or 64 x 64 CTA
tiles (gbd_problem.tile); both give the same bits (same k order, same
epilogue), so the choice is purely about speed: small and ragged problems waste
less work in 32 x 32 tiles, large ones keep more independent MMAs per warp in
64 x 64 tiles.  The tuner times both on synthetic batches of each size bucket
(bucket = floor(log2(sqrt(m*n))), i.e. the geometric mean of the output edges)
and records the faster one.  Every measurement goes through the library's own
grouped entry points; nothing here computes a GEMM.
"""
from __future__ import annotations

import json
import math
import os

from . import gbdgemm, synth

CANDIDATES = (32, 64)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gbdgemm", "tune.json")


def bucket_of(m: int, n: int) -> int:
    return int(math.floor(math.log2(max(1.0, math.sqrt(max(1, m) * max(1, n))))))


class Autotuner:
    """Per-bucket native tile choice, persisted in a JSON cache."""

    def __init__(self, cache_path: str | None = None):
        self.cache_path = cache_path or os.environ.get("GBD_TUNE_CACHE", DEFAULT_CACHE)
        self.table: dict[str, dict] = {}
        self.load()

    # --- cache ---
    def load(self) -> None:
        try:
            with open(self.cache_path) as f:
                data = json.load(f)
            self.table = data.get("native_tile", {})
        except (OSError, ValueError):
            self.table = {}

    def save(self) -> None:
        d = os.path.dirname(self.cache_path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump({"native_tile": self.table, "version": gbdgemm.gbd_version()}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    # --- lookup ---
    def tile_for(self, m: int, n: int, k: int = 0) -> int:
        """Tuned tile edge for an m x n output, or 0 (library default) when the bucket is untuned."""
        e = self.table.get(str(bucket_of(m, n)))
        return int(e["tile"]) if e else 0

    def apply(self, descriptors: list[dict]) -> list[dict]:
        """Fills the 'tile' field of native problem descriptors (dicts of gbd_problem fields)."""
        for d in descriptors:
            if d.get("mode", 0) == gbdgemm.GBD_MODE_NATIVE and not d.get("tile"):
                d["tile"] = self.tile_for(d["m"], d["n"], d.get("k", 0))
        return descriptors

    # --- measurement ---
    def tune_native_tiles(self, buckets=range(5, 12), per_bucket: int = 16, reps: int = 3, seed: int = 7) -> dict:
        """Times each candidate tile on a synthetic batch per bucket; returns and caches the table."""
        import torch
        dev = torch.device("cuda")
        for b in buckets:
            lo, hi = 2 ** b, 2 ** (b + 1) - 1
            sizes = synth.log_uniform_sizes(seed + b, per_bucket, lo, hi)
            ks = synth.log_uniform_sizes(seed + 100 + b, per_bucket, 32, 2048)[:, 2]
            probs, keep = [], []
            for i in range(per_bucket):
                m, n, k = int(sizes[i, 0]), int(sizes[i, 1]), int(ks[i])
                A = torch.from_numpy(synth.uniform_pm1(seed + 3 * i, m * k)).to(dev)
                B = torch.from_numpy(synth.uniform_pm1(seed + 3 * i + 1, k * n)).to(dev)
                C = torch.zeros(m * n, dtype=torch.float64, device=dev)
                keep += [A, B, C]
                probs.append(dict(transa="N", transb="N", mode=gbdgemm.GBD_MODE_NATIVE, m=m, n=n, k=k, alpha=1.0,
                                  beta=0.0, A=A, lda=m, B=B, ldb=k, C=C, ldc=m))
            flops = sum(2.0 * p["m"] * p["n"] * p["k"] for p in probs)
            timings = {}
            for tile in CANDIDATES:
                for p in probs:
                    p["tile"] = tile
                arr = gbdgemm.problem_array(probs)
                wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
                ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
                rc, plan = gbdgemm.gbd_grouped_plan_create(arr, ws, wsb)
                gbdgemm.check(rc)
                try:
                    gbdgemm.check(gbdgemm.gbd_grouped_plan_run(plan))  # warm-up
                    best = float("inf")
                    for _ in range(reps):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        gbdgemm.check(gbdgemm.gbd_grouped_plan_run(plan))
                        e1.record()
                        torch.cuda.synchronize()
                        best = min(best, e0.elapsed_time(e1))
                    timings[tile] = best
                finally:
                    gbdgemm.gbd_grouped_plan_destroy(plan)
            tile = min(timings, key=timings.get)
            self.table[str(b)] = {"tile": tile, "ms": {str(t): v for t, v in timings.items()},
                                  "tflops": flops / (timings[tile] / 1e3) / 1e12}
        self.save()
        return self.table
