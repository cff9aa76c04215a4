"""Exactness argument of the FP64-accurate tensor-core product, checked on CPU.

The refinement residual (and D^-1 of the mixed chain) computes complex products
y = sum_k a_k x_k to FP64 accuracy on bf16 tensor cores.  The scheme: every
operand v with |v| < 2^S (S = the frexp exponent bound of its matrix row or RHS
column) becomes T = trunc(|v| 2^(55-S)) < 2^55, written as eight balanced
base-128 digits d_0 .. d_7 (|d| <= 64, exact in bf16); the 36 digit products
with p + q <= 7 are summed per level L = p + q; within a window of 256 complex
inner rows every level sum stays an integer of magnitude <= 2^24, so FP32
accumulation in any order is exact; each window's levels are merged in int64
as V = (hi << 16) + (lo >> 12) and added to an FP64 sum as V 2^(E+F-49).

This module models that arithmetic with Python integers (it imports neither
the oracle nor the CUDA library) and checks, against exact rational
arithmetic:
  * the bias trick yields balanced digits that reconstruct trunc(|v| 2^(55-S));
  * no level sum of a window can exceed 2 * 256 * 32640 = 16 711 680 < 2^24
    (from the digit ranges; a constructed input of doubles reaches
    16 515 072), so no FP32 partial sum leaves the exact integers, and a
    window of 512 rows would not be safe;
  * the error of a whole product stays below the bound
      2^(E+F) (2K eps_t + n_win 2^-49) + 2^-52 (sum_w |y_w| + |y|),
    eps_t < 2^-52.5 per real product term (the dropped levels p + q >= 8,
    at most 7 * 4096 * 128^6 * 2^-110 + ..., plus the truncation of both
    operands, 2 * 2^-55), the second term the window merge (12 dropped bits),
    the third the FP64 roundings (int64 to double, one addition per window).
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

NS = 8                                    # digits per operand
BIAS = sum(64 * 128 ** m for m in range(7))
WIN = 256                                 # complex inner rows per exact window


def digits(v, S):
    """Balanced base-128 digits of trunc(|v| 2^(55-S)) with the sign of v,
    from the IEEE bit pattern (subnormals flush to zero)."""
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    e = (b >> 52) & 0x7FF
    U = 0
    if e != 0:
        M = (b & ((1 << 52) - 1)) | (1 << 52)
        sh = e - 1020 - S
        U = (M << sh) if sh >= 0 else (M >> -sh if -sh < 64 else 0)
    V = U + BIAS
    sg = -1 if b >> 63 else 1
    d = [sg * (V >> 49)] + [sg * (((V >> (49 - 7 * p)) & 0x7F) - 64) for p in range(1, NS)]
    return d, U


def scale_exp(vals):
    """Smallest S with |v| < 2^S for all v (frexp exponent of the largest)."""
    return max((math.frexp(v)[1] for v in vals if v != 0.0), default=-1021)


def eps_term():
    """Error of one real product term relative to 2^(E+F): the dropped digit
    levels 8..14 plus the truncation of both operands."""
    dropped = sum((15 - L) * 64 * 64 * Fraction(128) ** (14 - L) for L in range(8, 15))
    return dropped * Fraction(2) ** -110 + 2 * Fraction(2) ** -55


def product(A, x):
    """Model of one output row: y = A x for complex A (K,), x (K,), returned
    as (y, sum of |window partials|, max |level sum|, E, F, n_win)."""
    E = scale_exp([v for a in A for v in (a.real, a.imag)])
    F = scale_exp([v for z in x for v in (z.real, z.imag)])
    da = [(np.array(digits(a.real, E)[0]), np.array(digits(a.imag, E)[0])) for a in A]
    dx = [(np.array(digits(z.real, F)[0]), np.array(digits(z.imag, F)[0])) for z in x]
    out, wsum, lmax = [], [], 0
    for comp in (0, 1):                  # real, imaginary part of the output
        acc, ws = 0.0, Fraction(0)
        for w0 in range(0, len(A), WIN):
            lv = [0] * NS
            for k in range(w0, min(len(A), w0 + WIN)):
                (ar, ai), (xr, xi) = da[k], dx[k]
                pairs = [(xr, ar), (xi, -ai)] if comp == 0 else [(xr, ai), (xi, ar)]
                for xd, ad in pairs:
                    for L in range(NS):
                        lv[L] += int(sum(int(xd[p]) * int(ad[L - p]) for p in range(L + 1)))
            lmax = max(lmax, max(abs(t) for t in lv))
            hi = sum(lv[L] << (7 * (3 - L)) for L in range(4))
            lo = sum(lv[L] << (7 * (7 - L)) for L in range(4, NS))
            V = (hi << 16) + (lo >> 12)
            assert abs(V) < 2 ** 62
            part = Fraction(float(V)) * Fraction(2) ** (E + F - 49)   # int64 -> double
            ws += abs(part)
            acc = float(Fraction(acc) + part)                           # one FP64 rounding
        out.append(acc)
        wsum.append(ws)
    return complex(out[0], out[1]), wsum, lmax, E, F, (len(A) + WIN - 1) // WIN


def exact(A, x):
    re = sum(Fraction(a.real) * Fraction(z.real) - Fraction(a.imag) * Fraction(z.imag)
             for a, z in zip(A, x))
    im = sum(Fraction(a.imag) * Fraction(z.real) + Fraction(a.real) * Fraction(z.imag)
             for a, z in zip(A, x))
    return re, im


def check_bound(A, x):
    y, wsum, lmax, E, F, nw = product(A, x)
    assert lmax <= 2 ** 24
    ex = exact(A, x)
    for got, want, ws in zip((y.real, y.imag), ex, wsum):
        bound = (Fraction(2) ** (E + F) * (2 * len(A) * eps_term() + nw * Fraction(2) ** -49)
                 + Fraction(2) ** -52 * (ws + abs(want)))
        assert abs(Fraction(got) - want) <= bound, (float(abs(Fraction(got) - want)),
                                                    float(bound))
    return y


def test_bias_digits_are_balanced_and_exact():
    rng = np.random.default_rng(0)
    vals = list(rng.standard_normal(300) * 10.0 ** rng.uniform(-12, 12, 300))
    vals += [1.0, -1.0, 0.5, -0.75, 2.0 ** -30, -(2.0 - 2.0 ** -52), 1e-300, 5e-324, 0.0]
    for v in vals:
        for slack in (0, 1, 7):
            S = scale_exp([v]) + slack if v != 0.0 else 0
            d, U = digits(v, S)
            assert 0 <= abs(d[0]) <= 64 and all(-64 <= t <= 64 for t in d)
            assert all(-64 <= math.copysign(1, v) * t <= 63 for t in d[1:]) or v == 0.0
            want = math.floor(Fraction(abs(v)) * Fraction(2) ** (55 - S)) if abs(v) >= 2.0 ** -1022 else 0
            assert U == want and U < 2 ** 55
            sg = -1 if math.copysign(1, v) < 0 else 1
            assert sum(t * 128 ** (7 - p) for p, t in enumerate(d)) == sg * U


def level_max(L):
    """Largest |sum_{p+q=L} x_p a_q| over the digit ranges (d_0 in [0, 64],
    d_1..d_7 in [-64, 63] for a positive value, mirrored for a negative one),
    all products taking one sign."""
    lo = {0: (0, 64)}
    rng_of = lambda p: lo.get(p, (-64, 63))
    best = 0
    for sign in (1, -1):
        tot = 0
        for p in range(L + 1):
            (a0, a1), (b0, b1) = rng_of(p), rng_of(L - p)
            tot += max(sign * u * w for u in (a0, a1) for w in (b0, b1))
        best = max(best, tot)
    return best


def test_window_worst_case_fits_fp32():
    # upper bound from the digit ranges: level 7 with all products positive
    assert max(level_max(L) for L in range(NS)) == level_max(7) == 6 * 4096 + 2 * 64 * 63
    bound = 2 * WIN * level_max(7)               # 2 real terms per complex inner row
    assert bound == 16711680 < 2 ** 24
    # close to attained by doubles: at the top of the scale (|v| in [2^(S-1),
    # 2^S)) T = mantissa * 4, so d_7 is a multiple of 4; digits
    # [64, -64 x 6, 60] are a double's, with both real terms of the real
    # output part adding
    T = 64 * 128 ** 7 - 64 * sum(128 ** m for m in range(1, 7)) + 60
    vmax = math.ldexp(float(T), -55)
    assert int(float(T)) == T and digits(vmax, 0)[0] == [64] + [-64] * 6 + [60]
    A = np.full(WIN, complex(vmax, -vmax))
    x = np.full(WIN, complex(vmax, vmax))
    _, _, lmax, _, _, _ = product(A, x)
    assert lmax == 2 * WIN * (6 * 4096 + 2 * 64 * 60) == 16515072
    # so a window of 512 complex rows would not be safe
    assert 2 * (2 * WIN) * (6 * 4096 + 2 * 64 * 60) > 2 ** 24


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_product_error_within_bound(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(200, 600))                  # one to three windows, ragged
    A = (rng.standard_normal(K) * 10.0 ** rng.uniform(-4, 4, K)
         + 1j * rng.standard_normal(K) * 10.0 ** rng.uniform(-4, 4, K))
    x = rng.standard_normal(K) + 1j * rng.standard_normal(K) * 1e-3
    if seed == 3:                                    # one sign everywhere: no cancellation
        A = np.abs(A.real) + 1j * np.abs(A.imag)
        x = np.abs(x.real) + 0j
    y = check_bound(A, x)
    ref = complex(*(float(t) for t in exact(A, x)))
    assert abs(y - ref) <= 1e-12 * max(abs(ref), 1e-300) or seed != 3


def test_cancellation_is_absolute_not_relative():
    # a row whose products cancel: the bound is in units of 2^(E+F), so the
    # result may lose relative accuracy, exactly as FP64 dot products do
    K = 300
    rng = np.random.default_rng(7)
    a = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    A = np.concatenate([a, -a])
    x = np.ones(2 * K, complex)
    y = check_bound(A, x)
    assert abs(y) <= 2.0 ** (scale_exp([1.0]) + scale_exp(list(a.real) + list(a.imag))) * 2e-12
