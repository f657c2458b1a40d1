"""The double-word ("double-float") arithmetic the double-word inner COCG uses, restated in
numpy float32 (no GPU): the error-free transformations are exact and a 27-term Dot2-style
accumulation of products of double-word operands is accurate to about 2^-45 of sum |a x|, the
precision the design relies on (against 2^-24 for plain complex64).

Published sources of the algorithms: TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2), FastTwoSum
(Dekker 1971), TwoProd with a fused multiply-add, Dot2 (Ogita, Rump & Oishi 2005)."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def fma32(a, b, c):
    # exact a*b + c in float64 (products of two float32 are exact there), then one rounding
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def split(v):
    hi = f32(v)
    return hi, f32(np.float64(v) - np.float64(hi))


def dot2_dw(a, x):
    """sum a_i x_i for double-word a_i, x_i: head products exact (TwoProd), cross terms and all
    rounding errors into a separate float, TwoSum on the running head."""
    s, c = f32(0), f32(0)
    for (ah, al), (xh, xl) in zip(a, x):
        p = f32(ah * xh)
        e = fma32(ah, xh, -p)
        e = fma32(ah, xl, e)
        e = fma32(al, xh, e)
        s, t = two_sum(s, p)
        c = f32(c + f32(t + e))
    return fast_two_sum(s, c)


def exact(v):
    return Fraction(float(np.float64(v)))


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, b = f32(rng.standard_normal() * 10 ** rng.uniform(-5, 5)), f32(rng.standard_normal() * 10 ** rng.uniform(-5, 5))
        s, e = two_sum(a, b)
        assert exact(s) + exact(e) == exact(a) + exact(b)
        hi, lo = (a, b) if abs(a) >= abs(b) else (b, a)
        s, e = fast_two_sum(hi, lo)
        assert exact(s) + exact(e) == exact(a) + exact(b)
        p = f32(a * b)
        assert exact(p) + exact(fma32(a, b, -p)) == exact(a) * exact(b)


def test_split_keeps_about_48_bits():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(5000) * 10 ** rng.uniform(-8, 8, 5000)
    for x in v:
        hi, lo = split(x)
        assert abs(Fraction(float(x)) - exact(hi) - exact(lo)) <= Fraction(2) ** -48 * abs(Fraction(float(x)))


def test_dot2_of_27_double_word_products():
    rng = np.random.default_rng(2)
    worst_dw, worst_f32 = 0.0, 0.0
    for _ in range(300):
        a = rng.standard_normal(27)
        x = rng.standard_normal(27) * 10 ** rng.uniform(-3, 3, 27)
        ad, xd = [split(v) for v in a], [split(v) for v in x]
        h, l = dot2_dw(ad, xd)
        ref = sum((exact(ah) + exact(al)) * (exact(xh) + exact(xl)) for (ah, al), (xh, xl) in zip(ad, xd))
        scale = sum(abs(Fraction(float(p)) * Fraction(float(q))) for p, q in zip(a, x))
        worst_dw = max(worst_dw, float(abs(exact(h) + exact(l) - ref) / scale))
        s32 = f32(0)
        for p, q in zip(a, x):
            s32 = fma32(f32(p), f32(q), s32)
        worst_f32 = max(worst_f32, float(abs(Fraction(float(s32)) - ref) / scale))
    assert worst_dw <= 2.0 ** -44
    assert worst_f32 >= 2.0 ** -30  # plain float32 is some 2^14 less precise
