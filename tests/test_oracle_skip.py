"""Pins of the oracle's skip length (Algorithm 1: delta = floor(log r / log(1-p))).

The exact real floor has an integer characterisation that needs no
logarithm: delta = max{k >= 0 : (1-p)^k >= r}.  With p = Q/S and
r = (2a+1)/2^53 this is (S-Q)^k * 2^53 >= (2a+1) * S^k in exact integers,
which the tests evaluate with Python big integers.  Boundary cases put r on
the grid points adjacent to (1-p)^k, where x lies within ~2^-53 of an integer.
"""
import math

import numpy as np

import oracle


def exact_floor(a: int, Q: int, S: int, kmax: int) -> int:
    """max{k : (S-Q)^k 2^53 >= (2a+1) S^k}, capped at kmax."""
    num, den = 1, 1  # (S-Q)^k, S^k
    r_num = 2 * a + 1
    k = 0
    while k < kmax:
        num2, den2 = num * (S - Q), den * S
        if num2 * 2**53 >= r_num * den2:
            num, den, k = num2, den2, k + 1
        else:
            break
    return k


def r_of(a: int) -> float:
    return (2 * a + 1) * 2.0**-53


def test_skip_random_against_exact_integers():
    rng = np.random.default_rng(11)
    st = oracle.Stats()
    for _ in range(1500):
        S = int(rng.integers(2, 10**9))
        Q = int(rng.integers(1, S))
        a = int(rng.integers(0, 2**52))
        p = Q / S
        # keep x small enough for the big-integer loop
        if -math.log(r_of(a)) / -math.log1p(-p) > 400:
            continue
        R = 10**6
        assert oracle.skip(r_of(a), Q, S, R, st) == exact_floor(a, Q, S, R), (a, Q, S)


def _boundary_grid_points(Q: int, S: int, k: int):
    """Grid indices a whose r = (2a+1)/2^53 sit just below/above (1-p)^k."""
    num, den = (S - Q) ** k, S**k
    # (2a+1) <= num/den * 2^53  <=>  a <= (num*2^53/den - 1)/2
    t = (num * 2**53) // den
    a0 = (t - 1) // 2
    return [x for x in (a0 - 1, a0, a0 + 1, a0 + 2) if 0 <= x < 2**52]


def test_skip_near_integer_boundaries_exact():
    rng = np.random.default_rng(12)
    st = oracle.Stats()
    n = 0
    for _ in range(300):
        S = int(rng.integers(3, 10**7))
        Q = int(rng.integers(1, S))
        p = Q / S
        kmax = int(min(60, 36.0 / -math.log1p(-p)))
        if kmax < 1:
            continue
        k = int(rng.integers(1, kmax + 1))
        for a in _boundary_grid_points(Q, S, k):
            got = oracle.skip(r_of(a), Q, S, 10**6, st)
            assert got == exact_floor(a, Q, S, 10**6), (a, Q, S, k)
            n += 1
    assert n > 500
    # these cases sit within ~1 ulp of an integer: the double evaluation must defer
    assert st.fallbacks > 0
    assert st.unresolved == 0


def test_skip_exact_integer_dyadic_case():
    # p = 1/2, r = 2^-53: x = 53 exactly
    st = oracle.Stats()
    assert oracle.skip(2.0**-53, 1, 2, 1000, st) == 53
    assert st.unresolved == 1  # no finite window separates an exact integer
    assert exact_floor(0, 1, 2, 1000) == 53
    # one grid step above: x just below 53
    assert oracle.skip(3 * 2.0**-53, 1, 2, 1000) == exact_floor(1, 1, 2, 1000) == 51


def test_skip_clamps_at_remaining_length():
    # p tiny: x is huge, the skip is clamped at R
    assert oracle.skip(0.5, 1, 10**9, 1000) == 1000
    assert oracle.skip(r_of(0), 1, 10**12, 7) == 7
    # p near 1: x in (0, 2)
    S = 10**9
    for a in (0, 1, 2**40, 2**51, 2**52 - 1):
        assert oracle.skip(r_of(a), S - 1, S, 100) == exact_floor(a, S - 1, S, 100)


def test_skip_is_geometric():
    """P(delta >= k) = (1-p)^k (the skip is a geometric variate)."""
    rng = np.random.default_rng(13)
    S, Q = 1000, 37
    p = Q / S
    a = rng.integers(0, 2**52, 40000, dtype=np.uint64)
    d = np.array([oracle.skip(r_of(int(x)), Q, S, 10**9) for x in a])
    for k in (1, 5, 10, 20, 40, 80):
        emp = (d >= k).mean()
        th = (1 - p) ** k
        sd = math.sqrt(th * (1 - th) / len(d))
        assert abs(emp - th) < 5 * sd + 1e-9, (k, emp, th)


def test_quad_helpers_against_exact_rationals():
    # -ln(A/B) for dyadic ratios is k ln 2
    hi, lo = oracle.neglog_ratio_quad(1.0, 8.0)
    assert abs((hi + lo) - 3 * math.log(2)) < 1e-15
    hi, lo = oracle.skip_x_quad(2.0**-53, 1.0, 2.0)
    assert hi == 53.0 and abs(lo) < 1e-28
