"""The FP32-pair (double-word) building blocks of the MIXED32 field solve, against exact
host arithmetic (fractions of the binary values involved).

The right-hand side of Eq. (7), the E update and the Chebyshev solve's refinements run on
pairs h + l of FP32 numbers; their accuracy claims (47 significant bits; the sum and the
product within a few 2^-47 of the exact result, Joldes, Muller and Popescu 2017) are
checked here on values spread over many binades, signs, zeros and the integer range of
the fixed-point current.
"""
from fractions import Fraction

import numpy as np
import pytest

import paper_1412_2480_gb300 as pic

pytestmark = pytest.mark.gpu


def inputs(n=4096, seed=11):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))
    x[:8] = [0.0, 1.0, -1.0, 0.5 + 2.0**-30, 3.0, -1e-30, 1e30, 2.0**-120]
    d = rng.integers(-(2**62), 2**62, n, dtype=np.int64) >> rng.integers(0, 62, n)
    d[:4] = [0, 1, -1, 2**47 + 12345]
    return x, d


def F(v):
    return Fraction(float(v))


def test_pair_conversions_match_exact_values():
    x, d = inputs()
    out = pic.pic_dword_check(x, d).astype(np.float64)
    for i in range(x.size):
        h, l = F(out[i, 0]), F(out[i, 1])
        a = F(x[i])
        if abs(x[i]) >= 2.0**-80:  # below 2^-81 the pair flushes its low word
            assert abs(h + l - a) <= abs(a) * Fraction(1, 2**46), (x[i], h, l)
            assert abs(out[i, 1]) <= abs(out[i, 0]) * 2.0**-23  # normalised: |l| <= ulp(h)
        # FP32 rounding to nearest, ties to even, as numpy's cast
        if abs(x[i]) >= 2.0**-126 and abs(x[i]) < 3e38:
            assert np.float32(out[i, 2]) == np.float32(x[i]), (x[i], out[i, 2])
        # integer -> pair
        k = Fraction(int(d[i]))
        hk, lk = F(out[i, 3]), F(out[i, 4])
        assert abs(hk + lk - k) <= abs(k) * Fraction(1, 2**46), (d[i], hk, lk)
        # the FP64 join of the pair returns a to the pair's precision
        if abs(x[i]) >= 2.0**-80:
            assert abs(out[i, 9]) <= abs(x[i]) * 2.0**-46


def test_pair_sum_and_product_within_their_bounds():
    x, d = inputs(seed=12)
    out = pic.pic_dword_check(x, d).astype(np.float64)
    n = x.size
    for i in range(n):
        a, b = x[i], x[(i + 1) % n]
        if min(abs(a), abs(b)) < 2.0**-75 and (a != 0.0 and b != 0.0):
            continue  # tiny values: the pairs' low words and error terms leave FP32's normal range
        pa = F(out[i, 0]) + F(out[i, 1])
        pb = F(out[(i + 1) % n, 0]) + F(out[(i + 1) % n, 1])
        s = F(out[i, 5]) + F(out[i, 6])
        m = F(out[i, 7]) + F(out[i, 8])
        # sloppy pair sum: absolute error a few 2^-47 of the operands' magnitudes
        assert abs(s - (pa + pb)) <= (abs(pa) + abs(pb)) * Fraction(1, 2**45), (a, b)
        if abs(float(pa * pb)) > 2.0**-70:  # the product's error term stays a normal FP32 number
            assert abs(m - pa * pb) <= abs(pa * pb) * Fraction(1, 2**44), (a, b)


def test_pair_sum_is_exact_for_cancelling_operands():
    # x + (-x) and the residual-like cancellation b - Ax: the pair sum of two pairs whose
    # values differ by a few ulps of the pair is exact
    x = np.array([1.0 + 2.0**-40, -1.0, 3.25, -3.25 - 2.0**-44], dtype=np.float64)
    out = pic.pic_dword_check(x, np.zeros(4, dtype=np.int64)).astype(np.float64)
    assert F(out[0, 5]) + F(out[0, 6]) == Fraction(2) ** -40
    assert F(out[2, 5]) + F(out[2, 6]) == -Fraction(2) ** -44


def test_check_rejects_bad_arguments():
    with pytest.raises(ValueError):
        pic.pic_dword_check(np.zeros(3), np.zeros(2, dtype=np.int64))
