"""Host checks of two formulas the modular kernels rely on, restated exactly in integers.

1. Residues (the preparation's residue writer).  For each modulus p, the bytes of |A'|
   weighted by 256^d mod p are summed by two dp4a starting from 0x4B000000 + c,
   c = -2^23 mod p; read as FP32 that word is x = 2^23 + s' with x = |A'| (mod p).  Then
   q = rint(x * fl(1/p)) (one fma against 1.5 * 2^23, so round to nearest even) and
   r = x - p q.  The BF16 operand is exact only if |r| <= 256 and the product bound of
   the chunked FP32 sums needs |r| <= 128: checked here for every byte sum the kernel can
   form, with fl(1/p) the FP32 reciprocal and the rounding done in exact integers.
2. The reconstruction (k_mod_crt).  With W_l = M/p_l, c_l = W_l^-1 mod p_l and the parked
   residues r_l = C' mod p_l in [0, p_l): X = sum_l r_l (c_l W_l) is congruent to C' modulo M,
   the quotient estimate Qe = floor(sum_l r_l ceil(c_l 2^16/p_l) / 2^16 + 1/2) is the quotient of
   the symmetric representative or one more (and then X - Qe M <= -M/2), and X - Qe M is formed
   modulo 2^96 (at most 12 moduli, M < 2^95) or 2^128 from byte dot products: S_d = sum_l r_l
   (byte d of V_l) < 2^20, per 32-bit limb k A_k = S_4k + 2^8 S_4k+1 and B_k = S_4k+2 + 2^8 S_4k+3
   (below 2^29), limb k = A_k + (B_k-1 >> 16) (below 2^30) plus (B_k << 16 mod 2^32) plus the
   carry of limb k - 1 (at most one); the representative of (-M/2, M/2] must come out for every C'.
3. The reduction of one exact FP32 chunk (the product epilogue when k <= 1024).  A chunk sum v is
   an integer with |v| <= 2^24; q = rint(v fl(1/p)) comes from one fma against 1.5 2^23 (round to
   nearest even at unit spacing while the sum stays in [2^23, 2^24)), r = v - p q from one exact
   fma, and p is added to a negative r: the result must be v mod p in [0, p) for every v.
4. Triangle tiles (DSYRK's triangular product).  Tile t of a triangle of T x T tiles is
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


def _crt_constants(n: int):
    M = 1
    for p in MODULI[:n]:
        M *= p
    V, e = [], []
    for p in MODULI[:n]:
        W = M // p
        c = pow(W % p, -1, p)
        assert c * W < M
        V.append(c * W)
        e.append((c * 2 ** 16 + p - 1) // p)
    return M, V, e


def _crt_kernel(r, n, M, V, e):
    """The kernel's reconstruction, step by step in exact integers; returns C' modulo 2^(32 L)."""
    L = 3 if n <= 12 else 4
    mod = 2 ** (32 * L)
    S = [sum(rl * ((Vl >> (8 * d)) & 0xFF) for rl, Vl in zip(r, V)) for d in range(4 * L)]
    assert max(S) < 2 ** 20  # the byte dot products of up to 16 moduli
    x, carry, bprev = [], 0, 0
    for k in range(L):
        A = S[4 * k] + (S[4 * k + 1] << 8)
        B = S[4 * k + 2] + (S[4 * k + 3] << 8)
        assert A < 2 ** 29 and B < 2 ** 29
        a = A + (bprev >> 16)
        assert a < 2 ** 30
        t = a + ((B << 16) & 0xFFFFFFFF) + carry  # add.cc / addc on 32-bit words
        assert t < 2 ** 33
        x.append(t & 0xFFFFFFFF)
        carry, bprev = t >> 32, B
        assert carry <= 1
    X = sum(w << (32 * j) for j, w in enumerate(x))
    assert X == sum(rl * Vl for rl, Vl in zip(r, V)) % mod
    qh = sum(rl * (el >> 8) for rl, el in zip(r, e))
    qe = (qh << 8) + 2 ** 15 + sum(rl * (el & 0xFF) for rl, el in zip(r, e))
    assert max(e) < 2 ** 16 and qe < 2 ** 32  # the 32-bit estimate
    xm = (X - (qe >> 16) * M) % mod
    if ((xm + M // 2 - 1) % mod) >> (32 * L - 1):  # X - Qe M <= -M/2: one too many
        xm = (xm + M) % mod
    return xm, mod


@pytest.mark.parametrize("n", range(1, 17))
def test_reconstruction_gives_the_symmetric_representative(n):
    M, V, e = _crt_constants(n)
    assert M < (2 ** 95 if n <= 12 else 2 ** 127)
    rng = np.random.default_rng(n)
    half = M // 2
    values = [0, 1, -1, half, -half + 1, half - 1, -half + 2]
    values += [int(x) for x in rng.integers(0, 2 ** 62, 200)]
    values += [int(rng.integers(0, 2 ** 62)) * 2 ** 64 % M - half for _ in range(200)]
    for cp in values:
        cp = (cp + half - 1) % M - half + 1  # the representative of (-M/2, M/2]
        r = [cp % p for p in MODULI[:n]]
        X = sum(rl * Vl for rl, Vl in zip(r, V))
        Qn = (X - cp) // M
        Qe = (sum(rl * el for rl, el in zip(r, e)) + 2 ** 15) >> 16
        assert Qe == Qn or (Qe == Qn + 1 and X - Qe * M <= -half)
        got, mod = _crt_kernel(r, n, M, V, e)
        assert got == cp % mod


@pytest.mark.parametrize("n", [1, 12, 13, 16])
def test_reconstruction_at_the_largest_residues(n):
    # every residue p_l - 1: the largest limb sums and quotient estimate
    M, V, e = _crt_constants(n)
    r = [p - 1 for p in MODULI[:n]]
    X = sum(rl * Vl for rl, Vl in zip(r, V))
    cp = X % M
    cp = cp - M if cp > M // 2 else cp
    got, mod = _crt_kernel(r, n, M, V, e)
    assert got == cp % mod


@pytest.mark.parametrize("p", MODULI)
def test_single_chunk_reduction_for_every_chunk_sum(p):
    N, E = _f32_recip(p)
    magic = 3 * 2 ** 22  # 1.5 2^23
    step = 1 << 22
    for lo in range(-(1 << 24), (1 << 24) + 1, step):
        v = np.arange(lo, min(lo + step, (1 << 24) + 1), dtype=np.int64)
        prod = v * N  # v fl(1/p) = prod / 2^E exactly (|prod| < 2^48)
        q = prod >> E  # floor
        rem = prod - (q << E)
        half = 1 << (E - 1)
        q = q + ((rem > half) | ((rem == half) & ((q & 1) == 1)))  # round to nearest, ties to even
        # the fma's sum v fl(1/p) + 1.5 2^23 stays where FP32 numbers are the integers
        assert int((prod >> E).min()) + magic >= 2 ** 23 and int((prod >> E).max()) + 1 + magic < 2 ** 24
        r = v - p * q  # exact: an integer below 2^8 in magnitude
        assert int(np.abs(r).max()) < p
        out = r + p * (r < 0)
        assert int(out.min()) >= 0 and int(out.max()) < p
        assert np.array_equal(out, v % p)


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
