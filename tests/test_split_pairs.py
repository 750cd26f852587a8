"""The arithmetic of the mixed path's split-pair differences, checked on the
host against exact rational arithmetic.

The mixed path stores an FP64 value u as hi = u rounded to FP32 and lo =
(u - hi) rounded to FP32, and takes its stencil differences on these pairs
with FP32 operations:
  first difference   u+ - u-           = (hi+ - hi-) + (lo+ - lo-)
  second difference  u+ + u- - 2 u0    = (d+ + d-) + ((e+ + e-) + (lo+ + lo- - 2 lo0)),
where hi+- - hi0 = d+- + e+- exactly (Knuth's two-sum). The claim is that
each result is the exact difference up to a few FP32 roundings of the
result itself and terms of order 2^-48 |u|, the accuracy of an FP64
difference rounded once to FP32. This is checked below with numpy float32,
operation by operation, on neighbourhoods built to stress the claim: zero
crossings (the high parts are not within a factor of two, so the
subtraction is not exact), large constant offsets (the difference is tiny
against the values), steep gradients and extrema. Differences of values
rounded to FP32 fail the same bound."""
from fractions import Fraction

import numpy as np

F = np.float32
EPS32 = 2.0 ** -24


def split(u):
    hi = u.astype(np.float32)
    lo = (u - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def two_diff(a, b):
    s = F(a - b)
    bv = F(s - a)
    e = F(F(a - F(s - bv)) - F(b + bv))
    return s, e


def first_diff(up, um):
    (hp, lp), (hm, lm) = split(up), split(um)
    return F(F(hp - hm) + F(lp - lm))


def second_diff(up, um, u0):
    (hp, lp), (hm, lm), (h0, l0) = split(up), split(um), split(u0)
    dp, ep = two_diff(hp, h0)
    dm, em = two_diff(hm, h0)
    lo = F(F(lp + lm) - F(2.0) * l0)  # 2 lo0 is exact: the same as the kernel's fused multiply-add
    return F(F(dp + dm) + F(F(ep + em) + lo))


def exact(*terms):
    return float(sum((Fraction(float(c)) * Fraction(float(t)) for c, t in terms), Fraction(0)))


def cases(seed):
    """(u+, u-, u0) triples of FP64 values."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(400):
        kind = rng.integers(5)
        h = 10.0 ** rng.uniform(-3, -1)
        x0 = rng.uniform(-1, 1)
        if kind == 0:      # zero crossing of a smooth function
            f = lambda x: np.sin(7.0 * x) * 0.3
            x0 = rng.uniform(-0.01, 0.01)
        elif kind == 1:    # large constant offset
            c = 10.0 ** rng.uniform(2, 4) * rng.choice([-1, 1])
            f = lambda x, c=c: c + 1e-3 * np.cos(3.0 * x)
        elif kind == 2:    # steep gradient
            f = lambda x: np.tanh(40.0 * x)
        elif kind == 3:    # extremum: first differences cancel
            f = lambda x: 2.0 - np.cos(5.0 * x)
            x0 = rng.uniform(-1e-3, 1e-3)
        else:              # puncture-like 1/r
            f = lambda x: 1.0 + 0.5 / (abs(x) + 0.3)
        j = int(rng.integers(1, 4))
        out.append((f(x0 + j * h), f(x0 - j * h), f(x0)))
    return out


def test_first_difference_is_an_fp64_difference_rounded_to_fp32():
    for up, um, u0 in cases(1):
        got = float(first_diff(np.float64(up), np.float64(um)))
        want = exact((1, up), (-1, um))
        assert abs(got - want) <= 2.0 * EPS32 * abs(want) + 2.0 ** -46 * (abs(up) + abs(um)), (up, um)


def test_second_difference_is_an_fp64_difference_rounded_to_fp32():
    for up, um, u0 in cases(2):
        got = float(second_diff(np.float64(up), np.float64(um), np.float64(u0)))
        want = exact((1, up), (1, um), (-2, u0))
        assert abs(got - want) <= 2.0 * EPS32 * abs(want) + 2.0 ** -45 * (abs(up) + abs(um) + abs(u0)), (up, um, u0)


def test_two_diff_is_error_free():
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000)).astype(np.float32)
    b = (rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000)).astype(np.float32)
    for x, y in zip(a, b):
        s, e = two_diff(x, y)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(x)) - Fraction(float(y))


def test_values_rounded_to_fp32_miss_the_bound():
    """The bound above is not met by differencing FP32-rounded values: on
    the large-offset and extremum cases the error is many times the bar."""
    worst = 0.0
    for up, um, u0 in cases(2):
        naive = float(F(F(F(up) + F(um)) - F(2.0) * F(u0)))
        want = exact((1, up), (1, um), (-2, u0))
        bar = 2.0 * EPS32 * abs(want) + 2.0 ** -45 * (abs(up) + abs(um) + abs(u0))
        worst = max(worst, abs(naive - want) / bar)
    assert worst > 1e3
