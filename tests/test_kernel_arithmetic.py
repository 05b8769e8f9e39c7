"""Host checks of two formulas the modular kernels rely on, restated exactly in integers.

1. Residues (the preparation's residue writer).  For each modulus p, the bytes of |A'|
   weighted by 256^d mod p are summed by two dp4a starting from 0x4B000000 + c,
   c = -2^23 mod p; read as FP32 that word is x = 2^23 + s' with x = |A'| (mod p).  Then
   q = rint(x * fl(1/p)) (one fma against 1.5 * 2^23, so round to nearest even) and
   r = x - p q.  The BF16 operand is exact only if |r| <= 256 and the product bound of
   the chunked FP32 sums needs |r| <= 128: checked here for every byte sum the kernel can
   form, with fl(1/p) the FP32 reciprocal and the rounding done in exact integers.
2. Triangle tiles (DSYRK's triangular product).  Tile t of a triangle of T x T tiles is
   (r, c) with t = r (r + 1) / 2 + c, found from an FP32 square-root estimate corrected by
   integer steps; every tile that meets the triangle comes out exactly once.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]


def _f32_recip(p: int) -> tuple[int, int]:
    """fl32(1/p) as N / 2^E exactly."""
    inv = np.float32(1.0) / np.float32(p)
    mant, exp = math.frexp(float(inv))  # inv = mant 2^exp, mant in [0.5, 1)
    N = int(mant * 2 ** 24)
    E = 24 - exp
    assert N / 2 ** E == float(inv)
    return N, E


@pytest.mark.parametrize("p", MODULI)
def test_residue_in_range_for_every_byte_sum(p):
    N, E = _f32_recip(p)
    c = (p - (2 ** 23 % p)) % p
    assert (2 ** 23 + c) % p == 0
    s = np.arange(0, 8 * 255 * 255 + 1, dtype=np.int64)  # every sum of 8 bytes x weights < 256
    x = 2 ** 23 + c + s
    assert int(x.max()) < 2 ** 24  # the word 0x4B000000 + c + s still reads as 2^23 + c + s
    prod = x * N  # exact (< 2^48)
    q = prod >> E
    rem = prod - (q << E)
    half = 1 << (E - 1)
    q = q + ((rem > half) | ((rem == half) & ((q & 1) == 1)))  # round to nearest, ties to even
    r = x - p * q
    assert np.all((r - s) % p == 0)  # the residue class of s
    assert int(np.abs(r).max()) <= 128


def _tri_tile(t: int) -> tuple[int, int]:
    f32 = np.float32
    q = int((np.sqrt(f32(8.0) * f32(t) + f32(1.0)) - f32(1.0)) * f32(0.5))  # the kernel's FP32 estimate
    while (q + 1) * (q + 2) // 2 <= t:
        q += 1
    while q > 0 and q * (q + 1) // 2 > t:
        q -= 1
    return q, t - q * (q + 1) // 2


@pytest.mark.parametrize("T", [1, 2, 7, 32, 33, 100, 257])
def test_triangle_tiles_cover_the_triangle_once(T):
    seen = [_tri_tile(t) for t in range(T * (T + 1) // 2)]
    assert len(set(seen)) == len(seen)
    assert set(seen) == {(r, c) for r in range(T) for c in range(r + 1)}


def test_triangle_tiles_at_large_indices():
    # the FP32 estimate can be off for large t; the integer steps correct it
    for t in [2 ** 20 - 1, 2 ** 24 + 12345, 2 ** 30 - 7, 2 ** 31 - 1]:
        r, c = _tri_tile(t)
        assert 0 <= c <= r and r * (r + 1) // 2 + c == t
