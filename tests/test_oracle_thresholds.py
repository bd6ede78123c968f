"""Pin the oracle's Metropolis threshold tables against arbitrary-precision arithmetic.

Metropolis (Methods; SI section 1) accepts a move that raises the energy by dE > 0 with
probability exp(-dE / T).  The build draws a uniform 32-bit integer r32 and accepts iff
r32 < thr with thr = min(2^32 - 1, floor(2^32 exp(-beta dE))).  Viana-Bray: dE = 2m for
m = 1..d (Eq. 3, couplings +-1).  SK with binary couplings and the 1/sqrt(N) scale of Eq. 1:
dE = 2k / sqrt(N).  Here the same real numbers are evaluated with mpmath at 60 digits.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle

mpmath.mp.dps = 60
TWO32 = mpmath.mpf(2) ** 32


def exact_thr(x_double):
    """floor(2^32 exp(x)) clamped to 2^32-1, for the double x, plus a 'near an integer' flag."""
    v = TWO32 * mpmath.e ** mpmath.mpf(x_double)
    if v >= TWO32 - 1:
        return 0xFFFFFFFF, False
    f = int(mpmath.floor(v))
    near = (v - f) < mpmath.mpf("1e-6") or (f + 1 - v) < mpmath.mpf("1e-6")
    return f, near


def check_table(table, exponents):
    for idx, x in exponents:
        want, near = exact_thr(x)
        if near:
            assert abs(int(table[idx]) - want) <= 1
        else:
            assert int(table[idx]) == want, (idx, x)


@pytest.mark.parametrize("T", [0.6, 1.0, 1.2149, 1.8205, 3.0, 0.25])
def test_vb_thresholds_exact(T):
    dmax = 40
    thr = oracle.vb_thresholds(T, dmax)
    beta = 1.0 / T
    assert thr[0] == 0xFFFFFFFF
    check_table(thr, [(m, -2.0 * beta * m) for m in range(1, dmax + 1)])
    assert np.all(np.diff(thr.astype(np.int64)) <= 0), "table must be non-increasing in dE"


@pytest.mark.parametrize("T,N", [(0.4, 8192), (0.6, 512), (1.0, 1000), (2.0, 64)])
def test_sk_thresholds_exact(T, N):
    thr = oracle.sk_thresholds(T, N)
    beta = 1.0 / T
    ks = list(range(1, min(N, 400))) + list(range(N - 50, N))
    check_table(thr, [(k, -(2.0 * beta * k) / math.sqrt(N)) for k in ks if 1 <= k < N])
    assert np.all(np.diff(thr.astype(np.int64)) <= 0)


def test_zero_and_infinite_temperature_limits():
    assert np.all(oracle.vb_thresholds(0.0, 10)[1:] == 0)          # T = 0: never go uphill
    assert np.all(oracle.vb_thresholds(math.inf, 10) == 0xFFFFFFFF)  # T = inf: always
    assert np.all(oracle.sk_thresholds(0.0, 100)[1:] == 0)
    assert np.all(oracle.sk_thresholds(math.inf, 100) == 0xFFFFFFFF)


def test_acceptance_probability_matches_boltzmann_ratio():
    """thr / 2^32 equals exp(-beta dE) to within 2^-32 (the quantisation of the method)."""
    for T in (0.5, 1.0, 2.0):
        thr = oracle.vb_thresholds(T, 12)
        for m in range(1, 13):
            p = float(thr[m]) / 2**32
            assert abs(p - math.exp(-2.0 * m / T)) <= 2.0**-32 + 1e-15
