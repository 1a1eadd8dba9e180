"""Pins of the oracle's integer CDF tables against exact rational arithmetic.

The binomial table (integer Pascal recurrence, 2^63 fixed point) must agree
with floor(2^32 * CDF) of the exact Binomial(n, P/2^32) law to within one
unit; the Poisson table (double-precision recurrence) with floor(2^32 * CDF)
of the exact Poisson law (mpmath, 60 digits) to within one unit.
"""
from fractions import Fraction
from math import comb

import mpmath
import numpy as np
import pytest

import oracle as O


def exact_binomial_cdf_scaled(n, P):
    """floor(2^32 * P(X <= k)) for X ~ Binomial(n, P/2^32), k = 0..n-1, exactly."""
    Q = (1 << 32) - P
    out = []
    acc = 0
    for k in range(n):
        acc += comb(n, k) * P ** k * Q ** (n - k)
        out.append((acc << 32) // (1 << (32 * n)))
    return out


@pytest.mark.parametrize("p", [1e-9, 0.1, 0.2, 1.0 / 3.0, 0.5, 2.0 / 3.0, 0.9, 0.999])
def test_binomial_table_exact(p):
    P = O.quantise(p)
    T = O.binomial_table(P)
    for n in range(1, O.NMAX + 1):
        row = T[n * (n - 1) // 2: n * (n - 1) // 2 + n].astype(np.int64)
        ref = np.array(exact_binomial_cdf_scaled(n, P), dtype=object)
        diff = max(abs(int(a) - int(b)) for a, b in zip(row, ref))
        assert diff <= 1, (p, n, diff)
        assert np.all(np.diff(row) >= 0)
        assert row[-1] <= 0xFFFFFFFF


def test_binomial_table_extremes():
    # P = 1 (p = 2^-32) and P = 2^32 - 1 stay inside [0, 2^32 - 1]
    for P in (1, (1 << 32) - 1, 1 << 31):
        T = O.binomial_table(P).astype(np.int64)
        assert T.min() >= 0 and T.max() <= 0xFFFFFFFF
    # p = 1/2 is dyadic: every entry is exact
    T = O.binomial_table(1 << 31)
    for n in (1, 2, 5, 31, 63):
        row = T[n * (n - 1) // 2: n * (n - 1) // 2 + n]
        ref = exact_binomial_cdf_scaled(n, 1 << 31)
        assert [int(v) for v in row] == ref


def test_quantise_rule():
    assert O.quantise(0.0) == 0
    assert O.quantise(1.0) == 1 << 32
    assert O.quantise(0.5) == 1 << 31
    assert O.quantise(0.2) == 858993459  # floor(0.2 * 2^32 + 1/2)
    assert O.quantise(1.0 / 3.0) == 1431655765


@pytest.mark.parametrize("lam", [0.0, 1e-3, 0.5, 3.3333333333333335, 10.0, 30.0, 50.0, 123.4, 200.0, 650.0])
def test_poisson_table_exact(lam):
    T = O.poisson_table(lam).astype(np.int64)
    assert T[-1] == 0xFFFFFFFF
    if lam == 0.0:
        assert len(T) == 1  # a single entry: every draw gives 0
        return
    assert np.all(np.diff(T) >= 0)
    mpmath.mp.dps = 60
    lamx = mpmath.mpf(lam)
    acc = mpmath.mpf(0)
    term = mpmath.e ** (-lamx)
    for k in range(len(T) - 1):
        if k > 0:
            term = term * lamx / k
        acc += term
        ref = int(mpmath.floor(acc * 2 ** 32))
        assert abs(int(T[k]) - ref) <= 1, (lam, k, int(T[k]), ref)
    # the table ends where the exact tail mass beyond its last index is below ~2^-32
    k = len(T) - 1
    if k > 0:
        term = term * lamx / k
    acc += term
    tail = 1 - acc
    assert tail < mpmath.mpf(2) ** -31


def alias_induced_weights(thr, al, n):
    """Exact number of 32-bit draws u that the alias row n maps to each outcome:
    column j = u >> 26 (64 columns) covers [j 2^26, (j+1) 2^26); u < thr[j] gives j,
    else alias[j].  Outcomes above n must get no draw."""
    cols = O.ALIAS_COLS
    off = n * cols
    cnt = [0] * cols
    for j in range(cols):
        a0, a1 = j << 26, (j + 1) << 26
        t = int(thr[off + j])
        alias = int(al[off + j])
        if alias == j:
            cnt[j] += a1 - a0
        else:
            assert a0 <= t <= a1
            cnt[j] += t - a0
            cnt[alias] += a1 - t
    assert all(c == 0 for c in cnt[n + 1:]), (n, cnt[n + 1:])
    return cnt[:n + 1]


@pytest.mark.parametrize("p", [1e-9, 0.2, 1.0 / 3.0, 0.5, 0.9, 0.999])
def test_alias_table_realises_pmf_exactly(p):
    """Every draw u in [0, 2^32) is accounted for, and each outcome k of row n gets
    exactly W_k = T[n][k] - T[n][k-1] draws (the integer pmf of the CDF table)."""
    P = O.quantise(p)
    T = O.binomial_table(P).astype(np.int64)
    thr, al = O.alias_table(P)
    for n in range(0, O.NMAX + 1):
        if n == 0:
            W = [1 << 32]
        else:
            row = [int(v) for v in T[n * (n - 1) // 2: n * (n - 1) // 2 + n]]
            W = [row[0]] + [row[k] - row[k - 1] for k in range(1, n)] + [(1 << 32) - row[-1]]
        assert alias_induced_weights(thr, al, n) == W, (p, n)
