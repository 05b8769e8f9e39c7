"""Measured schedule selection for grouped native problems, cached as JSON.

The grouped FP64-MMA kernel can run each problem with 32 x 32 or 64 x 64 CTA
tiles (gbd_problem.tile) and with its inner dimension split into 2..16 parts per
output tile (gbd_problem.ksplit; the parts' sums are added in part order, so a
split is deterministic but rounds differently from the unsplit sum).  Small and
ragged outputs waste less work in 32 x 32 tiles, large ones keep more
independent MMAs per warp in 64 x 64 tiles; a small output with a deep k has few
tiles, each a long chain, and splitting k gives the persistent grid more items to
balance.  For emulated (split) problems the tile field names the kernel class:
128 the one-SM 128 x 128 kernel, 256 the two-SM 256 x 256 kernel (same bits
either way).  The tuner times the candidates on synthetic batches of each bucket
(output bucket = floor(log2(sqrt(m*n))), the geometric mean of the output edges;
k bucket = floor(log2(k))) and records the fastest.  Every measurement goes
through the library's own grouped entry points; nothing here computes a GEMM.
"""
from __future__ import annotations

import json
import math
import os

from . import gbdgemm, synth

CANDIDATES = (32, 64)
KSPLITS = (1, 2, 4, 8)
EMU_CLASSES = (128, 256)
# split k only where an output bucket has few tiles: edges up to 2^SPLIT_MAX_BUCKET
SPLIT_MAX_BUCKET = 8
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gbdgemm", "tune.json")


def bucket_of(m: int, n: int) -> int:
    return int(math.floor(math.log2(max(1.0, math.sqrt(max(1, m) * max(1, n))))))


def kbucket_of(k: int) -> int:
    return int(math.floor(math.log2(max(1, k))))


class Autotuner:
    """Per-bucket native tile choice, persisted in a JSON cache."""

    def __init__(self, cache_path: str | None = None):
        self.cache_path = cache_path or os.environ.get("GBD_TUNE_CACHE", DEFAULT_CACHE)
        self.table: dict[str, dict] = {}
        self.split_table: dict[str, dict] = {}
        self.emu_table: dict[str, dict] = {}
        self.load()

    # --- cache ---
    def load(self) -> None:
        try:
            with open(self.cache_path) as f:
                data = json.load(f)
            self.table = data.get("native_tile", {})
            self.split_table = data.get("native_ksplit", {})
            self.emu_table = data.get("emulated_class", {})
        except (OSError, ValueError):
            self.table = {}
            self.split_table = {}
            self.emu_table = {}

    def save(self) -> None:
        d = os.path.dirname(self.cache_path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump({"native_tile": self.table, "native_ksplit": self.split_table, "emulated_class": self.emu_table,
                       "version": gbdgemm.gbd_version()}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    # --- lookup ---
    def tile_for(self, m: int, n: int, k: int = 0) -> int:
        """Tuned tile edge for an m x n output, or 0 (library default) when the bucket is untuned."""
        e = self.table.get(str(bucket_of(m, n)))
        return int(e["tile"]) if e else 0

    def ksplit_for(self, m: int, n: int, k: int) -> int:
        """Tuned inner-dimension split for an m x n x k problem, or 1 when untuned."""
        e = self.split_table.get(f"{bucket_of(m, n)}_{kbucket_of(k)}")
        return int(e["ksplit"]) if e else 1

    def emulated_class_for(self, m: int, n: int, k: int) -> int:
        """Tuned kernel class (128 or 256) of an emulated m x n x k problem, or 0 (library default)."""
        e = self.emu_table.get(f"{bucket_of(m, n)}_{kbucket_of(k)}")
        return int(e["tile"]) if e else 0

    def apply(self, descriptors: list[dict]) -> list[dict]:
        """Fills the 'tile' and 'ksplit' fields of native problem descriptors, and the 'tile' (kernel
        class) of emulated ones, where they are left at 0 (dicts of gbd_problem fields)."""
        for d in descriptors:
            mode = d.get("mode", 0)
            if mode == gbdgemm.GBD_MODE_EMULATED:
                if not d.get("tile"):
                    d["tile"] = self.emulated_class_for(d["m"], d["n"], d.get("k", 0))
                continue
            if mode != gbdgemm.GBD_MODE_NATIVE:
                continue
            if not d.get("tile"):
                d["tile"] = self.tile_for(d["m"], d["n"], d.get("k", 0))
            if not d.get("ksplit"):
                d["ksplit"] = self.ksplit_for(d["m"], d["n"], d.get("k", 0))
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
                timings[tile] = self._time_batch(probs, reps)
            tile = min(timings, key=timings.get)
            self.table[str(b)] = {"tile": tile, "ms": {str(t): v for t, v in timings.items()},
                                  "tflops": flops / (timings[tile] / 1e3) / 1e12}
        self.save()
        return self.table

    def tune_native_ksplit(self, out_buckets=range(5, SPLIT_MAX_BUCKET + 1), k_buckets=range(9, 12),
                           per_bucket: int = 8, reps: int = 3, seed: int = 11) -> dict:
        """Times each split in KSPLITS on a synthetic batch per (output bucket, k bucket), with the
        tuned (or default) tile of the output bucket; returns and caches the table."""
        import torch
        dev = torch.device("cuda")
        for b in out_buckets:
            for kb in k_buckets:
                sizes = synth.log_uniform_sizes(seed + 17 * b + kb, per_bucket, 2 ** b, 2 ** (b + 1) - 1)
                ks = synth.log_uniform_sizes(seed + 1000 + 17 * b + kb, per_bucket, 2 ** kb, 2 ** (kb + 1) - 1)[:, 2]
                probs, keep = [], []
                for i in range(per_bucket):
                    m, n, k = int(sizes[i, 0]), int(sizes[i, 1]), int(ks[i])
                    A = torch.from_numpy(synth.uniform_pm1(seed + 5 * i, m * k)).to(dev)
                    B = torch.from_numpy(synth.uniform_pm1(seed + 5 * i + 1, k * n)).to(dev)
                    C = torch.zeros(m * n, dtype=torch.float64, device=dev)
                    keep += [A, B, C]
                    probs.append(dict(transa="N", transb="N", mode=gbdgemm.GBD_MODE_NATIVE, m=m, n=n, k=k, alpha=1.0,
                                      beta=0.0, A=A, lda=m, B=B, ldb=k, C=C, ldc=m, tile=self.tile_for(m, n)))
                timings = {}
                for ksplit in KSPLITS:
                    for p in probs:
                        p["ksplit"] = ksplit
                    timings[ksplit] = self._time_batch(probs, reps)
                best = min(timings, key=timings.get)
                self.split_table[f"{b}_{kb}"] = {"ksplit": best, "ms": {str(t): v for t, v in timings.items()}}
        self.save()
        return self.split_table

    def tune_emulated_class(self, out_buckets=range(8, 12), k_buckets=range(9, 12), per_bucket: int = 8,
                            reps: int = 2, seed: int = 13, slices: int = 7) -> dict:
        """Times the one-SM and two-SM kernel classes on a synthetic batch of split-emulated problems
        per (output bucket, k bucket) at a fixed slice count; returns and caches the table."""
        import torch
        dev = torch.device("cuda")
        for b in out_buckets:
            for kb in k_buckets:
                sizes = synth.log_uniform_sizes(seed + 17 * b + kb, per_bucket, 2 ** b, 2 ** (b + 1) - 1)
                ks = synth.log_uniform_sizes(seed + 1000 + 17 * b + kb, per_bucket, 2 ** kb, 2 ** (kb + 1) - 1)[:, 2]
                probs, keep = [], []
                for i in range(per_bucket):
                    m, n, k = int(sizes[i, 0]), int(sizes[i, 1]), int(ks[i])
                    A = torch.from_numpy(synth.uniform_pm1(seed + 5 * i, m * k)).to(dev)
                    B = torch.from_numpy(synth.uniform_pm1(seed + 5 * i + 1, k * n)).to(dev)
                    C = torch.zeros(m * n, dtype=torch.float64, device=dev)
                    keep += [A, B, C]
                    probs.append(dict(transa="N", transb="N", mode=gbdgemm.GBD_MODE_EMULATED, slices=slices, m=m, n=n,
                                      k=k, alpha=1.0, beta=0.0, A=A, lda=m, B=B, ldb=k, C=C, ldc=m))
                timings = {}
                for tile in EMU_CLASSES:
                    for p in probs:
                        p["tile"] = tile
                    timings[tile] = self._time_batch(probs, reps)
                best = min(timings, key=timings.get)
                self.emu_table[f"{b}_{kb}"] = {"tile": best, "ms": {str(t): v for t, v in timings.items()}}
        self.save()
        return self.emu_table

    @staticmethod
    def _time_batch(probs, reps: int) -> float:
        """Best device time (ms) of `reps` runs of one grouped plan over `probs`."""
        import torch
        arr = gbdgemm.problem_array(probs)
        wsb = gbdgemm.gbd_dgemm_grouped_workspace_size(arr)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
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
            return best
        finally:
            gbdgemm.gbd_grouped_plan_destroy(plan)
