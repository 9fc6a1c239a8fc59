"""The float-float arithmetic of the complex128 product's kernels, restated in
numpy float32 and checked against exact rational arithmetic (CPU).

The GPU kernels (MM_C128_FF, and the float-float Krylov basis) carry a value as
an unevaluated sum of two floats and build every sum from error-free
transformations: Dekker's exact product (the FMA returns the rounding error of
a float product) and Knuth's two-sum.  This file restates the same steps with
float32 numpy scalars (an FMA of float32 operands is exact in float64 before
its single rounding to float32, up to a rare double rounding in the last bit of
the low-order terms) and pins the error bounds the GPU tests rely on:

* the split x = hi + lo of a double leaves at most 2^-48 |x|;
* a dot product of K terms accumulated as (running sum, correction) is within
  a few 2^-48 sqrt(K) of sum |a b| (bound used: 2^-47 sqrt(K) sum |a b|; the
  worst of twelve seeded cases at K = 300 and 540 is 4.3e-14, against 1e-7 for
  plain FP32 accumulation);
* the renormalised sum and product of the FFT stages are within 2^-46 of the
  exact result, relative to |a| + |b| and |a b|.

These pin the method (the algorithm as the kernels state it), not the kernels;
the GPU tests compare the kernels' products with the FP64 product and the
oracle.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32


def split(x: float):
    hi = f32(x)
    lo = f32(x - float(hi))
    return hi, lo


def fma32(a, b, c):
    # exact product of two floats fits a double; one rounding to float32
    return f32(float(a) * float(b) + float(c))


def ff_mac(acc, ah, al, bh, bl):
    """acc += (ah + al)(bh + bl); acc = [s, c] as in the kernels' ff_mac."""
    s, c = acc
    p = f32(ah * bh)
    e = fma32(ah, bh, -p)
    t = f32(s + p)
    bb = f32(t - s)
    z = f32(f32(s - f32(t - bb)) + f32(p - bb))
    c = f32(c + f32(z + e))
    c = fma32(ah, bl, c)
    c = fma32(al, bh, c)
    return [t, c]


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def ffv_add(a, b):
    s, e = two_sum(a[0], b[0])
    e = f32(e + f32(a[1] + b[1]))
    h = f32(s + e)
    return h, f32(e - f32(h - s))


def ffv_mul(a, b):
    p = f32(a[0] * b[0])
    e = fma32(a[0], b[0], -p)
    e = fma32(a[0], b[1], e)
    e = fma32(a[1], b[0], e)
    h = f32(p + e)
    return h, f32(e - f32(h - p))


def exact(x) -> Fraction:
    return Fraction(float(x))


def test_split_error():
    rng = np.random.default_rng(1)
    for x in rng.standard_normal(200) * 10.0 ** rng.integers(-20, 20, 200):
        hi, lo = split(float(x))
        err = abs(Fraction(float(x)) - exact(hi) - exact(lo))
        assert err <= Fraction(2) ** -48 * abs(Fraction(float(x)))


def _dot_case(K, seed):
    """Relative error of the restated float-float dot product of K random terms."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(K)
    b = rng.standard_normal(K)
    acc = [f32(0), f32(0)]
    for x, y in zip(a, b):
        ah, al = split(float(x))
        bh, bl = split(float(y))
        acc = ff_mac(acc, ah, al, bh, bl)
    got = exact(acc[0]) + exact(acc[1])
    ref = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    mag = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b))
    return abs(got - ref) / mag


def test_dot_product_error_bound():
    """K = 300 (a macromodel row) and 540 (a near-field row): within 2^-47 sqrt(K) of
    sum |a b| (1.6e-13 at K = 540), about a millionth of plain FP32 accumulation's error."""
    for K in (300, 540):
        worst = max(_dot_case(K, s) for s in range(6))
        assert worst <= Fraction(2) ** -47 * Fraction(np.sqrt(K)), (K, float(worst))
    # and a plain float32 accumulation is far worse (the test would notice a dropped correction)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(540), rng.standard_normal(540)
    s = f32(0)
    for x, y in zip(a, b):
        s = fma32(f32(x), f32(y), s)
    ref = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    mag = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b))
    assert abs(exact(s) - ref) / mag > Fraction(2) ** -40


def test_renormalised_sum_and_product():
    rng = np.random.default_rng(5)
    for _ in range(300):
        x, y = rng.standard_normal(2) * 10.0 ** rng.integers(-3, 3, 2)
        a, b = split(float(x)), split(float(y))
        ea, eb = exact(a[0]) + exact(a[1]), exact(b[0]) + exact(b[1])
        s = ffv_add(a, b)
        assert abs(exact(s[0]) + exact(s[1]) - (ea + eb)) <= Fraction(2) ** -46 * (abs(ea) + abs(eb))
        assert abs(exact(s[1])) <= abs(exact(s[0])) * Fraction(2) ** -23   # renormalised
        p = ffv_mul(a, b)
        assert abs(exact(p[0]) + exact(p[1]) - ea * eb) <= Fraction(2) ** -46 * abs(ea * eb)
