"""Pins of the certified precision choice of the emulations (oracle/certify.c).

The choice is the smallest slice count s (split emulation) or integer bit count t (modular
emulation) whose a-priori truncation bound stays within the componentwise FP64 target on
every element, or the width at which every scaled entry is an integer.  These tests tie it
to things other than its own formula: the emulation models run at the chosen precision
against the Dot2 oracle's bound, exact integer products, hand-derived values for all-ones
operands, the structured input on which magnitude sums misjudge |A||B|, and a rational
evaluation on tiny problems.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

from conftest import U
from paper_1609_00076_gb300 import synth


def _within_bound(oracle_mod, out, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, tol):
    ref = oracle_mod.dgemm_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    G = oracle_mod.abs_bound_rows(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc)
    err = np.abs(out - ref)
    ok = err <= tol * G
    return bool(ok.all()), float(np.max(np.where(G > 0, err / np.where(G > 0, G, 1.0), 0.0)) / tol)


def test_all_ones_hand_values(oracle_mod):
    # op(A) = op(B) = ones, k = 1024: sigma = tau = 1, every scaled entry is 1/2, mu = nu = k/2,
    # G^ = k/4.  Modular: 2^(-t-1)(k + k 2^(-t-1)) <= (2k - 3) u k/4 first holds at t = 44
    # (t = 43 gives 2^-42 (1 + 2^-44) against 2045 2^-53 < 2^-42).  Split (one segment, r = 6):
    # 2^-7s 4 (1 + (s-1)(1 + 2^-7)) <= 2042 2^-53 first holds at s = 7 (s = 6 gives 2^-37.4).
    # Every scaled entry is an integer at one bit (1/2 * 2), so the choice is exact: t = 1, s = 1.
    m, n, k = 7, 5, 1024
    c = oracle_mod.certify("N", "N", m, n, k, np.ones(m * k), m, np.ones(k * n), k)
    assert (c["t_cert"], c["s_cert"], c["t_exact"], c["s_exact"]) == (44, 7, 1, 1)
    assert (c["t"], c["s"]) == (1, 1)
    assert c["moduli"] == oracle_mod.cert_moduli(1, k)
    assert c["rho"] == 4.0 and c["gamma"] == 4.0 / k
    out = oracle_mod.ozmod_dgemm_rows("N", "N", m, n, k, 1.5, np.ones(m * k), m, np.ones(k * n), k, 0.0, None, m,
                                      c["t"])
    assert np.all(out == 1.5 * k)
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.5, np.ones(m * k), m, np.ones(k * n), k, 0.0, None, m,
                                      c["s"])
    assert np.all(out == 1.5 * k)


def _v2(x: int) -> int:
    """2-adic valuation of a non-zero integer."""
    v = 0
    while x % 2 == 0:
        x //= 2
        v += 1
    return v


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_integer_inputs_exact_width(oracle_mod, ta, tb):
    m, n, k = 23, 19, 333
    ra, ca = (k, m) if ta == "T" else (m, k)
    rb, cb = (n, k) if tb == "T" else (k, n)
    A = synth.matrix("int8", ra, ca, ra, 31)
    B = synth.matrix("int8", rb, cb, rb, 32)
    Ai = synth.view(A, ra, ca, ra).astype(np.int64)
    Bi = synth.view(B, rb, cb, rb).astype(np.int64)
    Ai = Ai.T if ta == "T" else Ai
    Bi = Bi.T if tb == "T" else Bi
    # the width at which a row's scaled integers a 2^(t - sigma) are integers: sigma - v2(a)
    def width(rows):
        w = 0
        for r in rows:
            nz = [int(x) for x in r if x != 0]
            if not nz:
                continue
            sig = max(abs(x) for x in nz).bit_length()  # frexp exponent of an integer
            w = max(w, max(sig - _v2(abs(x)) for x in nz))
        return w
    tx = max(width(Ai), width(Bi.T))
    c = oracle_mod.certify(ta, tb, m, n, k, A, ra, B, rb)
    assert c["t_exact"] == tx
    dA, dB = (width(Ai) + 6) // 7, (width(Bi.T) + 6) // 7
    assert c["s_exact"] == max(1, dA + dB - 1)
    assert c["t"] == min(c["t_cert"], tx) and c["s"] == min(c["s_cert"], c["s_exact"])
    exact = (Ai @ Bi).astype(np.float64)
    out = oracle_mod.ozmod_dgemm_rows(ta, tb, m, n, k, 1.0, A, ra, B, rb, 0.0, None, m, c["t"])
    assert np.array_equal(out.reshape(n, m).T, exact)
    out = oracle_mod.ozaki_dgemm_rows(ta, tb, m, n, k, 1.0, A, ra, B, rb, 0.0, None, m, c["s"])
    assert np.array_equal(out.reshape(n, m).T, exact)


def _inputs(kind, ta, tb, m, n, k, seed):
    ra, ca = (k, m) if ta == "T" else (m, k)
    rb, cb = (n, k) if tb == "T" else (k, n)
    if kind.startswith("halves"):
        d = int(kind[6:])
        # op(A): its second half of the inner dimension scaled by 2^-d; op(B): its first half
        A = synth.matrix("uniform", ra, ca, ra, seed)
        va = A.reshape(ca, ra)  # storage columns
        if ta == "N":
            va[k // 2:, :] *= 2.0 ** -d
        else:
            va[:, k // 2:] *= 2.0 ** -d
        B = synth.matrix("uniform", rb, cb, rb, seed + 1)
        vb = B.reshape(cb, rb)
        if tb == "N":
            vb[:, : k // 2] *= 2.0 ** -d
        else:
            vb[: k // 2, :] *= 2.0 ** -d
        return A, ra, B, rb
    if kind == "sparse":
        A = synth.matrix("uniform", ra, ca, ra, seed)
        B = synth.matrix("uniform", rb, cb, rb, seed + 1)
        A[synth.coin(seed + 2, A.size, 0.7)] = 0.0
        B[synth.coin(seed + 3, B.size, 0.7)] = 0.0
        A.reshape(ca, ra)[:, 0] = 0.0  # a zero row (N) or column (T) of the storage
        return A, ra, B, rb
    e = {"uniform": 0, "e8": 8, "e32": 32}[kind]
    return synth.matrix("scaled", ra, ca, ra, seed, e), ra, synth.matrix("scaled", rb, cb, rb, seed + 1, e), rb


@pytest.mark.parametrize("kind", ["uniform", "e8", "e32", "halves4", "halves8", "sparse"])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("tol", [0.0, 1e-10])
def test_choice_meets_the_bound(oracle_mod, kind, ta, tb, tol):
    m, n, k = 37, 29, 700
    A, lda, B, ldb = _inputs(kind, ta, tb, m, n, k, 400 + len(kind))
    C0 = synth.matrix("uniform", m, n, m, 77)
    c = oracle_mod.certify(ta, tb, m, n, k, A, lda, B, ldb, tol)
    target = tol if tol > 0 else 2 * k * U
    assert c["t"] < 63 or c["s"] < 10, c
    if c["t"] < 63:
        out = oracle_mod.ozmod_dgemm_rows(ta, tb, m, n, k, -0.75, A, lda, B, ldb, 0.5, C0, m, c["t"])
        ok, worst = _within_bound(oracle_mod, out, ta, tb, m, n, k, -0.75, A, lda, B, ldb, 0.5, C0, m, target)
        assert ok, (c, worst)
    if c["s"] < 10:
        out = oracle_mod.ozaki_dgemm_rows(ta, tb, m, n, k, -0.75, A, lda, B, ldb, 0.5, C0, m, c["s"])
        ok, worst = _within_bound(oracle_mod, out, ta, tb, m, n, k, -0.75, A, lda, B, ldb, 0.5, C0, m, target)
        assert ok, (c, worst)


def test_structured_input_is_refused(oracle_mod):
    # rows of A: uniform on the first half of k, uniform * 2^-30 on the second; columns of B the
    # mirror image.  Every term of (|A||B|)_ij carries 2^-30, the magnitude sums do not.
    m = n = 64
    k = 1024
    A = synth.halves_matrix(m, k, m, 901, 30, small_cols_from=k // 2)
    B = synth.halves_matrix(k, n, k, 902, 30, small_rows_below=k // 2)
    c = oracle_mod.certify("N", "N", m, n, k, A, m, B, k)
    assert c["t"] == 63 and c["moduli"] == 0 and c["s"] == 10
    target = 2 * k * U
    # the estimate from magnitude sums picked 44 bits (8 slices): far outside the bound
    out = oracle_mod.ozmod_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, 44)
    ok, worst = _within_bound(oracle_mod, out, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, target)
    assert not ok and worst > 1e4
    # and the refusal is needed: the most bits 16 moduli allow at this k still miss it
    tmax = max(t for t in range(1, 63) if oracle_mod.cert_moduli(t, k))
    out = oracle_mod.ozmod_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, tmax)
    ok, worst = _within_bound(oracle_mod, out, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, target)
    assert not ok
    out = oracle_mod.ozaki_dgemm_rows("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, 9)
    ok, _ = _within_bound(oracle_mod, out, "N", "N", m, n, k, 1.0, A, m, B, k, 0.0, None, m, target)
    assert not ok


def test_zero_blocks_need_nothing(oracle_mod):
    # block-diagonal operands: the off-diagonal blocks of |A||B| are exactly zero and carry no
    # requirement, so the whole matrix needs what its diagonal blocks need
    h, k2 = 12, 300
    m = n = 2 * h
    k = 2 * k2
    A = np.zeros(m * k)
    B = np.zeros(k * n)
    Av, Bv = A.reshape(k, m), B.reshape(n, k)
    X1 = synth.values("uniform", 1, h * k2).reshape(k2, h)
    X2 = synth.values("scaled", 2, h * k2, 8).reshape(k2, h)
    Y1 = synth.values("uniform", 3, k2 * h).reshape(h, k2)
    Y2 = synth.values("scaled", 4, k2 * h, 8).reshape(h, k2)
    Av[:k2, :h], Av[k2:, h:] = X1, X2
    Bv[:h, :k2], Bv[h:, k2:] = Y1, Y2
    c = oracle_mod.certify("N", "N", m, n, k, A, m, B, k)
    c1 = oracle_mod.certify("N", "N", h, h, k2, X1.ravel().copy(), h, Y1.ravel().copy(), k2,
                            tol=2 * k * U)
    c2 = oracle_mod.certify("N", "N", h, h, k2, X2.ravel().copy(), h, Y2.ravel().copy(), k2,
                            tol=2 * k * U)
    # the blocks' k is half the whole one's: compare at the whole problem's target (both have
    # one segment).  The split rule's dropped-pair term counts the whole k, zeros included, so
    # the whole problem may need one slice more than its blocks
    assert c["t_cert"] == max(c1["t_cert"], c2["t_cert"])
    assert max(c1["s_cert"], c2["s_cert"]) <= c["s_cert"] <= max(c1["s_cert"], c2["s_cert"]) + 1


def test_rational_evaluation_on_tiny_problems(oracle_mod):
    # the rule evaluated in exact rationals on tiny problems, with loose targets where the
    # k 2^(-t-1) and (s-1) k terms matter
    rng = np.random.default_rng(11)
    for trial in range(40):
        m, n, k = int(rng.integers(1, 4)), int(rng.integers(1, 4)), int(rng.integers(1, 6))
        A = np.ldexp(rng.integers(-255, 256, m * k).astype(np.float64), rng.integers(-12, 3, m * k))
        B = np.ldexp(rng.integers(-255, 256, k * n).astype(np.float64), rng.integers(-12, 3, k * n))
        tol = float(rng.choice([1e-3, 1e-6, 0.05]))
        c = oracle_mod.certify("N", "N", m, n, k, A, m, B, k, tol)

        def frexp_e(x):
            return int(np.frexp(x)[1])
        sig = [max((frexp_e(A[p * m + i]) for p in range(k) if A[p * m + i] != 0), default=0) for i in range(m)]
        tau = [max((frexp_e(B[j * k + p]) for p in range(k) if B[j * k + p] != 0), default=0) for j in range(n)]
        ah = [[abs(Fraction(float(A[p * m + i]))) / Fraction(2) ** sig[i] for p in range(k)] for i in range(m)]
        bh = [[abs(Fraction(float(B[j * k + p]))) / Fraction(2) ** tau[j] for p in range(k)] for j in range(n)]
        ftol = Fraction(tol)
        u = Fraction(1, 2 ** 53)
        t_need, s_need = 1, 1
        for i in range(m):
            for j in range(n):
                G = sum(ah[i][p] * bh[j][p] for p in range(k))
                if G == 0:
                    continue
                mn = sum(ah[i]) + sum(bh[j])
                t = 1
                while t <= 62 and not (Fraction(1, 2 ** (t + 1)) * (mn + k * Fraction(1, 2 ** (t + 1)))
                                       <= (ftol - 3 * u) * G):
                    t += 1
                s = 1
                while s <= 9 and not (Fraction(1, 2 ** (7 * s)) * (mn + (s - 1) * (1 + Fraction(1, 128)) * k)
                                      <= (ftol - 6 * u) * G):
                    s += 1
                t_need, s_need = max(t_need, t), max(s_need, s)
        assert (c["t_cert"], c["s_cert"]) == (t_need, s_need), (trial, c, t_need, s_need)


def _moduli_products():
    mods = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]
    out, p = [], 1
    for q in mods:
        p *= q
        out.append(p)
    return out


def test_cauchy_schwarz_moduli_hand_values(oracle_mod):
    # all-ones rows of k = 1024: every scaled entry is 1/2, alpha^2 = beta^2 = k/4 = 256, and
    # A'B' = k (2^(t-1))^2 = 2^(2t + 8) exactly, the Cauchy-Schwarz bound (2^t 16 + 16)^2 with it.
    # At t = 42: 2 k 2^(2t) = 2^95 needs 13 moduli (12 multiply to 2^94.80); twice the
    # Cauchy-Schwarz bound, 2^93 (1 + 2^-42)^2, needs 12 (11 give 2^87.04)
    k = 1024
    c = oracle_mod.certify("N", "N", 3, 3, k, np.ones(3 * k), 3, np.ones(k * 3), k)
    assert c["alpha2"] == 256.0 and c["beta2"] == 256.0
    assert oracle_mod.cert_moduli(42, k) == 13
    assert oracle_mod.cert_moduli_cs(42, k, 256.0, 256.0) == 12
    P = _moduli_products()
    assert P[10] < 2 * k * 2 ** 82 < P[11]  # the exact |A'B'| needs the 12th modulus
    # rows of full magnitude (alpha^2 = beta^2 = k) leave the bound k 2^(2t)
    for t in (10, 30, 44):
        assert oracle_mod.cert_moduli_cs(t, 4096, 4096.0, 4096.0) == oracle_mod.cert_moduli(t, 4096)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_cauchy_schwarz_moduli_cover_the_exact_products(oracle_mod, seed):
    # brute force: the integers A'_ip = rn(a^_ip 2^t), B'_pj = rn(b^_pj 2^t) in exact arithmetic,
    # their product in Python integers; the chosen moduli must multiply to more than 2 max |A'B'|
    rng = np.random.default_rng(seed)
    m, n, k = 6, 5, 37
    kind = seed % 4
    A = rng.uniform(-1, 1, (m, k))
    B = rng.uniform(-1, 1, (k, n))
    if kind == 1:  # one large entry per row, the rest small: small square sums
        A *= 2.0 ** -12
        A[np.arange(m), rng.integers(0, k, m)] = 0.75
    elif kind == 2:  # powers of two over a wide range
        A *= 2.0 ** rng.integers(-20, 3, (m, k))
        B *= 2.0 ** rng.integers(-20, 3, (k, n))
    elif kind == 3:  # full-magnitude rows
        A = np.sign(A) * 0.999
        B = np.sign(B) * 0.999
    Acm = np.asfortranarray(A).ravel(order="F")
    Bcm = np.asfortranarray(B).ravel(order="F")
    c = oracle_mod.certify("N", "N", m, n, k, Acm, m, Bcm, k)

    def scaled(rowvals):
        e = int(max(np.frexp(v)[1] for v in rowvals if v != 0))
        return [Fraction(float(v)) / Fraction(2) ** e for v in rowvals]

    As = [scaled(A[i, :]) for i in range(m)]
    Bs = [scaled(B[:, j]) for j in range(n)]
    a2 = max(sum(x * x for x in r) for r in As)
    b2 = max(sum(x * x for x in r) for r in Bs)
    assert abs(c["alpha2"] - float(a2)) <= 1e-15 * float(a2)
    assert abs(c["beta2"] - float(b2)) <= 1e-15 * float(b2)
    P = _moduli_products()
    fewer = []
    for t in (3, 8, 20, 31, 45):
        Ai = [[round(x * 2 ** t) for x in r] for r in As]
        Bi = [[round(x * 2 ** t) for x in r] for r in Bs]
        cmax = max(abs(sum(a * b for a, b in zip(Ai[i], Bi[j]))) for i in range(m) for j in range(n))
        nm = oracle_mod.cert_moduli_cs(t, k, c["alpha2"], c["beta2"])
        assert nm >= 1 and P[nm - 1] > 2 * cmax, (t, nm)
        assert nm <= oracle_mod.cert_moduli(t, k)
        fewer.append(nm < oracle_mod.cert_moduli(t, k))
    if kind == 1:  # small square sums: fewer moduli than the k 2^(2t) bound somewhere
        assert any(fewer)
