"""The three-way bf16 split of the complex64 tensor-core chain, checked on CPU.

Both operands of the complex64 products are split as v = s0 + s1 + s2 with
s0 = bf16(v), s1 = bf16(v - s0), s2 = bf16(v - s0 - s1) (round to nearest
even; the differences are exact in FP32), and the six slice products
s_p t_q with p + q <= 2 are accumulated in FP32.  This module models the split
with NumPy bit operations (the standard round-to-nearest-even of a float32 to
its upper 16 bits; it imports neither the oracle nor the CUDA library) and
checks that the split is exact for every finite float32 tried down to 2^-100
(below, bf16's subnormal spacing 2^-133 bounds the loss) and that the dropped
products (p + q >= 3) cost less than 2^-22 of |v t| per product.
"""
import numpy as np


def bf16_rn(v):
    """float32 -> nearest bf16 (ties to even), returned as float32."""
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split3(v):
    v = np.asarray(v, np.float32)
    s0 = bf16_rn(v)
    r = (v - s0).astype(np.float32)
    s1 = bf16_rn(r)
    s2 = bf16_rn((r - s1).astype(np.float32))
    return s0, s1, s2


def finite_float32(rng, n):
    bits = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    v = bits.view(np.float32)
    v = v[np.isfinite(v)]
    # keep clear of the overflow edge (a bf16 rounding up of the largest
    # float32s would leave the finite range)
    return v[np.abs(v) < np.float32(3.0e38)]


def test_bf16_rounding_model():
    # exact cases: bf16 values map to themselves; halfway cases go to even
    assert bf16_rn(np.float32(1.0)) == 1.0
    one_ulp = np.float32(2.0 ** -7)                    # bf16 ulp of 1
    assert bf16_rn(np.float32(1.0) + one_ulp / 2) == 1.0              # tie -> even
    assert bf16_rn(np.float32(1.0) + 3 * one_ulp / 2) == 1.0 + 2 * one_ulp
    assert bf16_rn(np.float32(1.0) + one_ulp / 2 + np.float32(2.0 ** -20)) == 1.0 + one_ulp


def test_three_slices_reconstruct_every_float32():
    rng = np.random.default_rng(11)
    v = finite_float32(rng, 200000)
    v = np.concatenate([v, np.float32([1.0, -1.0, 1e-38, -1e-45, 3.3e38, 0.0,
                                       np.nextafter(np.float32(1.0), np.float32(2.0))])])
    s0, s1, s2 = split3(v)
    # summed in double (exact: the slices hold disjoint bit ranges)
    rec = s0.astype(np.float64) + s1.astype(np.float64) + s2.astype(np.float64)
    err = np.abs(rec - v.astype(np.float64))
    # exact while the third slice stays above bf16's subnormal spacing 2^-133;
    # below |v| ~ 2^-110 the lowest bits are lost, at most 2^-133 absolute
    big = np.abs(v) >= np.float32(2.0 ** -100)
    assert big.sum() > 0.85 * len(v)               # uniform bit patterns: ~89 %
    assert np.all(err[big] == 0.0)
    assert err.max() <= 2.0 ** -133


def test_six_slice_products_error():
    rng = np.random.default_rng(12)
    n = 100000
    v = (rng.standard_normal(n) * 10.0 ** rng.uniform(-5, 5, n)).astype(np.float32)
    t = (rng.standard_normal(n) * 10.0 ** rng.uniform(-5, 5, n)).astype(np.float32)
    a, b = split3(v), split3(t)
    six = sum(a[p].astype(np.float64) * b[q].astype(np.float64)
              for p in range(3) for q in range(3) if p + q <= 2)
    exact = v.astype(np.float64) * t.astype(np.float64)
    rel = np.abs(six - exact) / np.abs(exact)
    assert rel.max() < 2.0 ** -22
