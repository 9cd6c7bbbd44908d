"""The rounding inequality behind the search's exact pruning bound, checked on IEEE binary16.

The search sums T non-negative terms in fp16 (round to nearest even), each term first rounded
up to an fp16 value, and drops a pair only when that sum is below a threshold scaled for
rounding.  The inequality it relies on is

    exact sum  <=  fp16 sum * (1 + 2^-11)^T  +  T * 2^-25

(relative error of at most u/(1+u), u = 2^-11, per normal addition, and at most half the smallest
subnormal spacing, 2^-25, per subnormal one).  This file checks that inequality with numpy's
binary16 on random and adversarial sequences.  It is a property of the number format; it shares
nothing with the CUDA code.
"""
import math

import numpy as np
import pytest

U = 2.0 ** -11
SUB = 2.0 ** -25


def round_up_f16(x):
    """The smallest binary16 value >= x (x >= 0; above the range: +inf)."""
    with np.errstate(over="ignore"):
        h = np.float16(x)
    if float(h) < x:
        h = np.nextafter(h, np.float16(np.inf))
    return h


def f16_sum(terms):
    """Sequential binary16 sum with one rounding per addition (the two operands are added
    exactly in float64, then rounded to binary16)."""
    s = np.float16(0.0)
    with np.errstate(over="ignore"):
        for t in terms:
            s = np.float16(float(s) + float(t))
    return s


def check(terms):
    terms = [float(t) for t in terms]
    T = len(terms)
    s = f16_sum([round_up_f16(t) for t in terms])
    exact = math.fsum(terms)
    bound = float(s) * (1.0 + U) ** T + T * SUB
    assert exact <= bound, (T, exact, float(s), bound)
    return exact, float(s)


def test_round_up_is_the_next_value_at_or_above():
    rng = np.random.default_rng(0)
    for x in np.concatenate([rng.uniform(0, 70000, 2000), 2.0 ** rng.uniform(-30, 16, 2000)]):
        h = round_up_f16(x)
        assert float(h) >= x
        below = np.nextafter(h, np.float16(0))
        assert float(below) < x or float(h) == 0.0
    assert np.isinf(round_up_f16(65520.0)) and float(round_up_f16(65504.0)) == 65504.0
    assert float(round_up_f16(2.0 ** -26)) == 2.0 ** -24       # below the smallest subnormal


@pytest.mark.parametrize("seed", range(6))
def test_random_sequences(seed):
    rng = np.random.default_rng(seed)
    for _ in range(300):
        T = int(rng.integers(1, 129))
        kind = seed % 3
        if kind == 0:
            terms = rng.exponential(0.5, T)                      # noise: nu^2 of N(0,1), psi > 0
        elif kind == 1:
            terms = 2.0 ** rng.uniform(-30, 8, T)                # across the subnormal range
        else:
            terms = np.where(rng.random(T) < 0.1, rng.uniform(50, 400, T),
                             rng.exponential(0.5, T))             # a few bright epochs
        check(terms)


def test_adversarial_sequences():
    # every addition after the first loses almost half an ulp: the relative bound is tight
    for big in (2048.0, 1024.0, 16.0):
        half_ulp = big * 2.0 ** -11
        terms = [big] + [half_ulp * (1 - 2 ** -8)] * 127
        exact, s = check(terms)
        assert s == big and exact > big                          # the small terms were lost
    # terms far below the smallest subnormal: each rounds up to 2^-24, nothing is lost
    exact, s = check([2.0 ** -40] * 128)
    assert s >= exact
    # a sum that overflows is +inf and bounds anything
    _, s = check([60000.0, 60000.0] + [1.0] * 10)
    assert math.isinf(s)


def test_two_row_block_term_bounds_both_rows():
    # a block stores max(round_up(a), round_up(b)) = round_up(max(a, b)) (rounding up is
    # monotone), which is >= either row's term, so the block sum bounds both rows' sums
    rng = np.random.default_rng(7)
    a, b = rng.exponential(0.5, 1000), rng.exponential(0.5, 1000)
    for x, y in zip(a, b):
        m = max(round_up_f16(x), round_up_f16(y))
        assert m == round_up_f16(max(x, y)) and float(m) >= x and float(m) >= y
