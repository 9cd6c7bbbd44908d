"""The exact filters the evaluations apply before sorting a lightcurve (search_kernel: the thread
path's order statistics among the 8 largest and 8 smallest values; the warp and half-warp paths'
sample-checked candidates) drop a pair only through an upper bound ub on the sigma-G clip's upper
limit median + n sigma_G (Section 3.1, Eqs. 3-5): every epoch the clip keeps must lie at or below
ub.  These tests restate the two rules' index arithmetic (in float64) and check them against the
FP64 oracle's clip on random lightcurves: with outliers, ties, few epochs, and the quantile pairs
and widths the paper leaves to the user.  The kernels evaluate the same rules in float32 with a
rounding margin; their results are checked against the oracle by the GPU parity tests."""
import math

import numpy as np

import oracle

M = 8          # largest / smallest values the thread path keeps
SAMPLE = 32    # epochs in the warp paths' sample


def _ranks(n, q):
    h = (n - 1) * q
    return int(math.floor(h))


def thread_rule_ub(a, q_lo, q_mid, q_hi, n_sigma):
    n = len(a)
    s = np.sort(a)
    top = s[::-1][:M]
    bot = s[:M]
    u_mid = min(_ranks(n, q_mid) + 1, n - 1)
    u_hi = min(_ranks(n, q_hi) + 1, n - 1)
    l_lo = _ranks(n, q_lo)
    v_mid = top[min(n - u_mid, M) - 1]
    v_hi = top[min(n - u_hi, M) - 1]
    v_lo = bot[min(l_lo, M - 1)]
    c = oracle.sigma_g_coeff(q_lo, q_hi)
    return v_mid + n_sigma * (c * (v_hi - v_lo))


def sample_rule_ub(a, q_lo, q_mid, q_hi, n_sigma):
    n = len(a)
    samp = np.sort(a[:SAMPLE])
    m = len(samp)
    if m < 16:
        return math.inf
    i_lo = max(0, int(q_lo * (m - 1)) - 3)
    i_mid = min(m - 1, int(q_mid * (m - 1)) + 4)
    i_hi = min(m - 1, int(q_hi * (m - 1)) + 4)
    v_lo, v_mid, v_hi = samp[i_lo], samp[i_mid], samp[i_hi]
    c_lo = int((a < v_lo).sum())
    c_mid = int((a <= v_mid).sum())
    c_hi = int((a <= v_hi).sum())
    if not (c_lo <= _ranks(n, q_lo) and c_mid >= min(_ranks(n, q_mid) + 2, n)
            and c_hi >= min(_ranks(n, q_hi) + 2, n)):
        return math.inf
    c = oracle.sigma_g_coeff(q_lo, q_hi)
    return v_mid + n_sigma * (c * (v_hi - v_lo))


def _lightcurve(rng, n):
    kind = rng.integers(4)
    if kind == 0:
        a = rng.normal(size=n)
    elif kind == 1:                      # noise plus a few bright epochs (a crossed mover, spikes)
        a = rng.normal(size=n)
        k = rng.integers(1, 4)
        a[rng.choice(n, size=min(k, n), replace=False)] += rng.uniform(3, 30, size=min(k, n))
    elif kind == 2:                      # heavy ties
        a = rng.integers(-3, 4, size=n).astype(np.float64)
    else:                                # per-epoch noise levels differing fivefold (flux curve)
        a = rng.normal(size=n) * rng.uniform(1, 5, size=n)
    return a


QUANTILES = [(0.25, 0.5, 0.75, 2.0), (0.10, 0.50, 0.90, 1.5), (0.20, 0.45, 0.80, 2.5),
             (0.05, 0.5, 0.95, 3.0)]


def _check(rule, n_values, cases):
    rng = np.random.default_rng(2109)
    checked = tight = 0
    for _ in range(cases):
        n = int(rng.choice(n_values))
        a = _lightcurve(rng, n)
        q_lo, q_mid, q_hi, ns = QUANTILES[rng.integers(len(QUANTILES))]
        keep, med, sg = oracle.sigma_g_clip(a, q_lo, q_mid, q_hi, ns)
        ub = rule(a, q_lo, q_mid, q_hi, ns)
        hi_b = med + ns * sg
        assert ub >= hi_b - 1e-12 * max(1.0, abs(hi_b)), (n, q_lo, q_mid, q_hi, ub, hi_b)
        assert np.all(a[keep] <= ub + 1e-12 * max(1.0, abs(ub)))
        checked += 1
        tight += bool(ub < np.max(a))  # the bound excludes at least the largest value
    return checked, tight


def test_thread_rule_bounds_the_clip():
    checked, tight = _check(thread_rule_ub, [1, 2, 3, 5, 8, 9, 13, 15, 16, 20, 26, 31, 32],
                            4000)
    assert checked == 4000
    assert tight > 1000          # and it is not vacuous: it often excludes the brightest epoch


def test_sample_rule_bounds_the_clip():
    checked, tight = _check(sample_rule_ub, [33, 40, 45, 64, 80, 100, 127, 128], 3000)
    assert checked == 3000
    assert tight > 500           # about a quarter of the cases carry bright epochs


def test_thread_rule_order_statistics_at_the_ranks():
    """With n = 26 and the paper's quartiles the rule takes exactly the upper neighbours of the
    q_mid and q_hi ranks' order statistics where they fall among the 8 largest values, and the
    q_lo rank's own order statistic."""
    a = np.arange(26, dtype=np.float64)          # sorted value = rank
    c = oracle.sigma_g_coeff(0.25, 0.75)
    # q_hi: h = 18.75 -> upper neighbour rank 19 (7th largest); q_mid: h = 12.5 -> rank 13 lies
    # below the 8 largest, so the 8th largest (rank 18) bounds it; q_lo: h = 6.25 -> lower rank
    # 6, the 7th smallest value
    want = 18 + 2.0 * (c * (19 - 6))
    assert abs(thread_rule_ub(a, 0.25, 0.5, 0.75, 2.0) - want) < 1e-12
