"""CPU model of the exact-digit scheme that the tensor-core Gram matrices and rotations use: each
FP64 operand row (column) is cut under a common exponent E (|x| < 2^E) into
Y = trunc(x 2^(49-E)) = c0 2^42 + c1 2^35 + ... + c6 (c0 signed 8-bit, the others 7-bit), and only
the digit products of level s + t <= 6 are kept. These tests check, with exact rational
arithmetic, the two claims the kernels rest on: the accumulation of one level over K <= 146 terms
is exact in FP32 (below 2^24), and the result is within about 2^-46 of |x|max |w|max per term."""
from fractions import Fraction
import math

import numpy as np

NS, BITS, LEVELS = 7, 7, 6


def row_exponent(v):
    """E with |x| < 2^E for every x of the row (the kernels take it from the largest exponent)."""
    m = max(abs(float(x)) for x in v)
    return math.frexp(m)[1] if m > 0 else 0


def digits(x, E):
    Y = int(Fraction(float(x)) * Fraction(2) ** (49 - E))   # truncation toward zero
    c = [Y >> 42] + [(Y >> (42 - BITS * s)) & 127 for s in range(1, NS)]
    assert sum(cs << (42 - BITS * s) for s, cs in enumerate(c)) == Y
    return c


def digit_dot(x, w, levels=LEVELS):
    Ex, Fw = row_exponent(x), row_exponent(w)
    cx = [digits(a, Ex) for a in x]
    cw = [digits(b, Fw) for b in w]
    acc = [0] * (2 * NS - 1)                 # integer accumulator per level d = s + t
    for a, b in zip(cx, cw):
        for s in range(NS):
            for t in range(NS):
                acc[s + t] += a[s] * b[t]
    total = sum(Fraction(acc[d]) * Fraction(2) ** (84 - BITS * d) for d in range(levels + 1))
    return total * Fraction(2) ** (Ex + Fw - 98), acc, Ex, Fw


def exact_dot(x, w):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, w))


def test_one_level_accumulates_exactly_in_fp32_up_to_146_terms():
    # |c0| <= 128, c1..c6 <= 127: a product is at most 2^14, a level holds at most 7 products
    worst_level = 7 * 128 * 128
    assert worst_level * 146 < 2 ** 24 <= worst_level * 147
    rng = np.random.default_rng(5)
    x = -np.abs(rng.standard_normal(146))        # all negative: the largest leading digits
    w = -np.abs(rng.standard_normal(146))
    _, acc, _, _ = digit_dot(x, w)
    assert max(abs(a) for a in acc[:LEVELS + 1]) < 2 ** 24


def test_error_is_about_2_to_minus_46_of_the_maxima_per_term():
    # truncation leaves < 2^-48 of |x|max per operand value and the dropped levels d >= 7 about as
    # much again: measured 2^-46.7 .. 2^-47.8 per term on these draws; the test allows 2^-45
    rng = np.random.default_rng(7)
    worst = 0.0
    for K in (64, 128, 146, 64, 128, 146):
        x = rng.standard_normal(K) * np.exp2(rng.integers(-20, 20, K))   # spread magnitudes
        w = rng.standard_normal(K) * np.exp2(rng.integers(-20, 20, K))
        got, _, _, _ = digit_dot(x, w)
        err = abs(float(got - exact_dot(x, w)))
        scale = K * np.max(np.abs(x)) * np.max(np.abs(w))
        worst = max(worst, err / scale)
        assert err <= 2.0 ** -45 * scale
    assert 0.0 < worst


def test_dropping_a_kept_level_breaks_the_bound():
    # the kept levels are needed: stopping at level 5 leaves about 2^-40 per term
    rng = np.random.default_rng(11)
    x, w = rng.standard_normal(64), rng.standard_normal(64)
    got, _, _, _ = digit_dot(x, w, levels=5)
    err = abs(float(got - exact_dot(x, w)))
    assert err > 2.0 ** -43 * 64 * np.max(np.abs(x)) * np.max(np.abs(w))
