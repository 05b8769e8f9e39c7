"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws numbers: it holds none of the GEMM arithmetic, and both
the CUDA path and the CPU oracle receive its arrays as plain inputs.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; the 64-bit finaliser constants of Vigna's
public-domain splitmix64.c), evaluated counter-style:  x_i = mix(seed + (i+1)*gamma).

Value recipes (all values are dyadic and exact in FP64):
* uniform[-1,1):   2 * (x >> 11) * 2^-53 - 1
* small integers:  uniform on {lo..hi} via x mod (hi-lo+1)
* scaled uniform:  uniform[-1,1) * 2^U, U uniform on the integers {-e..e}

Matrices are column-major with a leading dimension ``ld >= rows`` (the BLAS
layout of the paper, Section 2.1); padding rows hold a NaN sentinel so that a
kernel that reads or writes outside the matrix is caught.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# NaN with a recognisable payload, used for padding rows and guard bands
SENTINEL_BITS = np.uint64(0x7FF8DEADBEEF0001)
SENTINEL = SENTINEL_BITS.view(np.float64)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 started at ``seed``, counters offset+1 .. offset+n."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n values uniform on [-1, 1), exact dyadic doubles."""
    z = splitmix64(seed, n)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def small_ints(seed: int, n: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """n integers uniform on {lo..hi}, as doubles."""
    z = splitmix64(seed, n)
    span = np.uint64(hi - lo + 1)
    return (z % span).astype(np.int64).astype(np.float64) + float(lo)


def scaled_uniform(seed: int, n: int, e: int) -> np.ndarray:
    """uniform[-1,1) * 2^U with U uniform on the integers {-e..e} (e >= 0)."""
    u = uniform_pm1(seed, n)
    if e == 0:
        return u
    z = splitmix64(seed ^ 0x5DEECE66D, n)
    ex = (z % np.uint64(2 * e + 1)).astype(np.int64) - e
    return np.ldexp(u, ex.astype(np.int32))


def values(kind: str, seed: int, n: int, e: int = 0) -> np.ndarray:
    if kind == "uniform":
        return uniform_pm1(seed, n)
    if kind == "int8":
        return small_ints(seed, n, -8, 8)
    if kind == "scaled":
        return scaled_uniform(seed, n, e)
    if kind == "ones":
        return np.ones(n, dtype=np.float64)
    raise ValueError(f"unknown value kind {kind!r}")


def colmajor(rows: int, cols: int, ld: int, vals: np.ndarray | None = None,
             pad: float = SENTINEL) -> np.ndarray:
    """A flat column-major buffer of ld*cols doubles holding a rows x cols
    matrix (vals given column by column); the ld-rows padding holds ``pad``."""
    if ld < max(1, rows):
        raise ValueError("ld < rows")
    buf = np.full(ld * max(cols, 0), pad, dtype=np.float64)
    if rows and cols:
        v = buf.reshape(cols, ld)
        v[:, :rows] = (np.zeros(rows * cols) if vals is None else vals).reshape(cols, rows)
    return buf


def matrix(kind: str, rows: int, cols: int, ld: int, seed: int, e: int = 0,
           pad: float = SENTINEL) -> np.ndarray:
    """Seeded column-major matrix (rows x cols, leading dimension ld)."""
    return colmajor(rows, cols, ld, values(kind, seed, rows * cols, e), pad)


def halves_matrix(rows: int, cols: int, ld: int, seed: int, d: int, small_cols_from: int | None = None,
                  small_rows_below: int | None = None, pad: float = SENTINEL) -> np.ndarray:
    """Seeded uniform[-1,1) matrix with one part scaled by 2^-d: the columns from
    ``small_cols_from`` on, or the rows below ``small_rows_below``.  With A (m x k) scaled on
    its second half of columns and B (k x n) on its first half of rows, every term of
    (|A||B|)_ij has one factor scaled down, while each row of A and column of B keeps
    entries near its largest: the case where magnitude sums misjudge |A||B|."""
    buf = matrix("uniform", rows, cols, ld, seed, pad=pad)
    v = buf.reshape(max(cols, 1), ld) if rows and cols else None
    if v is not None:
        if small_cols_from is not None:
            v[small_cols_from:, :rows] *= 2.0 ** -d
        if small_rows_below is not None:
            v[:, :small_rows_below] *= 2.0 ** -d
    return buf


def view(buf: np.ndarray, rows: int, cols: int, ld: int) -> np.ndarray:
    """The rows x cols matrix inside a column-major buffer, as a 2-D numpy view."""
    return buf[: ld * cols].reshape(cols, ld)[:, :rows].T


def seed_for(config_index: int, rep: int = 0) -> int:
    """Seed convention: configuration index * 1000 + repetition."""
    return config_index * 1000 + rep


def log_uniform_sizes(seed: int, count: int, lo: int = 32, hi: int = 2048) -> np.ndarray:
    """count x 3 integers (m, n, k), each log-uniform on [lo, hi]."""
    z = splitmix64(seed, 3 * count)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    v = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.floor(v + 0.5), lo, hi).astype(np.int64).reshape(count, 3)


def coin(seed: int, count: int, p: float = 0.5) -> np.ndarray:
    """count booleans, each True with probability p."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) < p


def exponential(seed: int, count: int, rate: float) -> np.ndarray:
    """count exponential inter-arrival gaps with the given rate (Poisson process)."""
    z = splitmix64(seed, count)
    u = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    return -np.log(u) / rate
