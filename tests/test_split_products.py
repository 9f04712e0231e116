"""CPU pin of the split-product arithmetic behind the tensor-core FP64 block products (the Ozaki
scheme: Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012), independent of the GPU code:
the method is restated here in exact integer arithmetic and its stated error bound is checked
against exact rational products on adversarial inputs (wide exponent ranges, one large entry
among tiny ones, near-total cancellation, integers).

op1 (V Y, contraction over K): every row of V is cut, relative to its largest binary exponent,
into seven 8-bit digits of its 56-bit aligned significand (sign-magnitude), every column of Y
likewise; the digit products of weight classes g = i + j <= 6 are summed exactly (as the FP32
accumulators do for at most 258 products of 8-bit digits), T = sum_g D_g 2^(48 - 8 g) is taken
without its 12 lowest bits and truncated once to FP64.  Stated bound:
    |result - exact| <= 2^-49 (K + 1) max_c |V[r][c]| max_c |Y[c][q]| + 2^-52 |exact|.
op3 (V^T W, contraction over rows): the same per 128-row tile with column exponents; the tile's
seven slices are added exactly and rounded once.  Stated bound per tile:
    2^-50 * 128 * max|V[., c]| * max|W[., q]| over the tile's rows (plus FP64 sums of tiles).
"""
from fractions import Fraction
import math

import numpy as np
import pytest


def _fields(x):
    """(sign, biased exponent field, 53-bit significand with the implicit bit) of a double;
    exponent 0 (zero, subnormal) reads as zero, as in the kernels."""
    u = int(np.float64(x).view(np.uint64))
    s = -1 if u >> 63 else 1
    e = (u >> 52) & 0x7FF
    m = (u & ((1 << 52) - 1)) | (1 << 52) if e else 0
    return s, e, m


def _digits(x, emax):
    """Sign and the seven digits of x's significand aligned to the exponent field emax."""
    s, e, m = _fields(x)
    sh = emax - e
    if e == 0 or sh > 52:
        return s, [0] * 7
    m56 = (m << 3) >> sh
    return s, [(m56 >> (8 * (6 - i))) & 0xFF for i in range(7)]


def _to_double_trunc(t, scale_exp):
    """t * 2^scale_exp truncated toward zero to FP64 (zero below the normal range)."""
    if t == 0:
        return 0.0
    sign = -1.0 if t < 0 else 1.0
    a = abs(t)
    nb = a.bit_length()
    if nb > 53:                                   # keep the 53 leading bits (truncation)
        a >>= nb - 53
        scale_exp += nb - 53
    top = a.bit_length() - 1 + scale_exp          # exponent of the leading bit
    if top < -1022:
        return 0.0 * sign
    if top > 1023:
        return sign * math.inf
    return sign * math.ldexp(float(a), scale_exp)


def op1_split(V, Y):
    n, K = V.shape
    N = Y.shape[1]
    out = np.zeros((n, N))
    fq = [max(_fields(Y[c, q])[1] for c in range(K)) for q in range(N)]
    ydig = [[_digits(Y[c, q], fq[q]) for q in range(N)] for c in range(K)]
    for r in range(n):
        er = max(_fields(V[r, c])[1] for c in range(K))
        vdig = [_digits(V[r, c], er) for c in range(K)]
        for q in range(N):
            D = [0] * 7
            for c in range(K):
                sv, dv = vdig[c]
                sy, dy = ydig[c][q]
                for i in range(7):
                    for j in range(7 - i):
                        D[i + j] += sv * dv[i] * sy * dy[j]
            T = sum(D[g] << (48 - 8 * g) for g in range(7))
            t = T >> 12                                    # floor, as the kernels' shifts
            out[r, q] = _to_double_trunc(t, er + fq[q] - 2108 + 12) if er and fq[q] else 0.0
    return out


def op3_split_tile(V, W):
    """One 128-row tile of V^T W (rows <= 128)."""
    KV, bw = V.shape[1], W.shape[1]
    ev = [max(_fields(V[r, c])[1] for r in range(V.shape[0])) for c in range(KV)]
    ew = [max(_fields(W[r, q])[1] for r in range(W.shape[0])) for q in range(bw)]
    G = np.zeros((KV, bw))
    for c in range(KV):
        vd = [_digits(V[r, c], ev[c]) for r in range(V.shape[0])]
        for q in range(bw):
            wd = [_digits(W[r, q], ew[q]) for r in range(W.shape[0])]
            total = 0
            for i in range(7):
                Ti = 0
                for j in range(7):
                    Dij = sum(vd[r][0] * vd[r][1][i] * wd[r][0] * wd[r][1][j] for r in range(V.shape[0]))
                    Ti += Dij << (48 - 8 * j)
                total += (Ti >> 12) << (48 - 8 * i)            # slices summed exactly
            G[c, q] = _to_double_trunc(total, ev[c] + ew[q] - 2108 + 12 - 48) if ev[c] and ew[q] else 0.0
    return G


def _exact(A, B):
    return [[sum(Fraction(float(A[r, c])) * Fraction(float(B[c, q])) for c in range(A.shape[1]))
             for q in range(B.shape[1])] for r in range(A.shape[0])]


def _cases(seed):
    rng = np.random.default_rng(seed)
    n, K, N = 24, 32, 4
    V = rng.standard_normal((n, K)) * 10.0 ** rng.uniform(-150, 150, (n, 1))
    V[0] = 1e-30
    V[0, 5] = 1e30                                           # one large entry among tiny ones
    V[1] = 2.0 ** rng.integers(-60, 60, K)                   # powers of two
    V[2] = rng.integers(-1000, 1001, K).astype(np.float64)   # integers
    Y = rng.standard_normal((K, N))
    Y[:, 1] *= 1e-200                                        # a tiny column
    # near-total cancellation in row 3: y = c - (V c) / ... built so that V[3] . Y[:, 2] ~ 0
    Y[:, 2] = rng.standard_normal(K)
    V[3] = rng.standard_normal(K)
    V[3, -1] = -(V[3, :-1] @ Y[:-1, 2]) / Y[-1, 2]
    return V, Y


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_op1_split_products_within_stated_bound(seed):
    V, Y = _cases(seed)
    got = op1_split(V, Y)
    ex = _exact(V, Y)
    K = V.shape[1]
    for r in range(V.shape[0]):
        for q in range(Y.shape[1]):
            e = ex[r][q]
            err = abs(Fraction(got[r, q]) - e)
            bound = (Fraction(2) ** -49 * (K + 1) * Fraction(float(np.abs(V[r]).max()))
                     * Fraction(float(np.abs(Y[:, q]).max())) + Fraction(2) ** -52 * abs(e)
                     + Fraction(2) ** -1022)
            assert err <= bound, (r, q, float(err), float(bound))


def test_op1_integers_exact():
    """Integer entries whose products fit 53 bits come out exact (the dropped classes hold
    only zero digits and the 12 dropped bits of T are zero)."""
    rng = np.random.default_rng(8)
    V = rng.integers(-1000, 1001, (16, 32)).astype(np.float64)
    Y = rng.integers(-1000, 1001, (32, 3)).astype(np.float64)
    got = op1_split(V, Y)
    assert np.array_equal(got, (V.astype(np.int64) @ Y.astype(np.int64)).astype(np.float64))


def test_op1_dropping_a_class_breaks_the_bound():
    """The pin is sensitive: keeping classes g <= 5 only (a dropped term) exceeds the bound on
    N(0,1) data, so a kernel that lost a class would be caught by these checks."""
    rng = np.random.default_rng(4)
    V = rng.standard_normal((8, 32))
    Y = rng.standard_normal((32, 2))
    K = 32
    worst = 0.0
    for r in range(8):
        er = max(_fields(V[r, c])[1] for c in range(K))
        for q in range(2):
            fq = max(_fields(Y[c, q])[1] for c in range(K))
            D = [0] * 7
            for c in range(K):
                sv, dv = _digits(V[r, c], er)
                sy, dy = _digits(Y[c, q], fq)
                for i in range(7):
                    for j in range(6 - i):                    # class 6 missing
                        D[i + j] += sv * dv[i] * sy * dy[j]
            T = sum(D[g] << (48 - 8 * g) for g in range(7))
            got = _to_double_trunc(T >> 12, er + fq - 2108 + 12)
            e = sum(Fraction(float(V[r, c])) * Fraction(float(Y[c, q])) for c in range(K))
            bound = (Fraction(2) ** -49 * (K + 1) * Fraction(float(np.abs(V[r]).max()))
                     * Fraction(float(np.abs(Y[:, q]).max())) + Fraction(2) ** -52 * abs(e))
            worst = max(worst, float(abs(Fraction(got) - e) / bound))
    assert worst > 1.0


def test_op3_tile_within_stated_bound():
    rng = np.random.default_rng(6)
    rows, KV, bw = 128, 6, 2
    V = rng.standard_normal((rows, KV)) * 10.0 ** rng.uniform(-50, 50, (1, KV))
    W = rng.standard_normal((rows, bw))
    V[7, 2] = 1e40
    G = op3_split_tile(V, W)
    ex = _exact(V.T.copy(), W)
    for c in range(KV):
        for q in range(bw):
            err = abs(Fraction(G[c, q]) - ex[c][q])
            bound = (Fraction(2) ** -50 * 128 * Fraction(float(np.abs(V[:, c]).max()))
                     * Fraction(float(np.abs(W[:, q]).max())) + Fraction(2) ** -52 * abs(ex[c][q])
                     + Fraction(2) ** -1022)
            assert err <= bound, (c, q, float(err), float(bound))


def test_fp16_digit_encoding_constants():
    """The FP16 digit encoding of the tensor-core kernels, checked against IEEE binary16: the
    bit pattern 0x6400 | d is 1024 + d for every digit d in [0, 255]; 0x3C00 / 0xBC00 are +1 / -1;
    XOR with 0xD800 turns +-1 into -+1024; and (1024 + d) s + (-1024 s) = s d exactly, so one
    FP16 FMA per digit gives the signed digit (products of two digits, at most 255^2, and sums of
    up to 258 of them are exact in the FP32 accumulator: 258 * 255^2 < 2^24)."""
    d = np.arange(256, dtype=np.uint16)
    enc = (np.uint16(0x6400) | d).view(np.float16)
    assert np.array_equal(enc.astype(np.float64), 1024.0 + d)
    for sbits, sval in ((0x3C00, 1.0), (0xBC00, -1.0)):
        s = np.array([sbits], dtype=np.uint16).view(np.float16)[0]
        c = np.array([sbits ^ 0xD800], dtype=np.uint16).view(np.float16)[0]
        assert float(s) == sval and float(c) == -1024.0 * sval
        # each step is exact in binary16 (|values| <= 1279 < 2^11), so the FMA equals this
        prod = (enc * s).astype(np.float64)
        assert np.array_equal(prod, (1024.0 + d) * sval)
        out = (enc * s + c).astype(np.float64)
        assert np.array_equal(out, sval * d)
    assert 258 * 255 ** 2 < 2 ** 24 < 259 * 255 ** 2      # 258 is the largest safe count
