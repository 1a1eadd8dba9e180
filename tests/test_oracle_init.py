"""Pins of the oracle's Poisson initial state (Sec. V: occupation numbers are
Poisson numbers with mean w_i P(rho), P(rho) = N^ave [1 + sin(2 pi x / L)]).

Checked against the Poisson law itself (chi-square of the histogram), the
stated means (per column of a sine profile), and the special cases that fix
the two initial-condition readings: with per-velocity weighting the means sum
to rho(x) over the velocities; without it every velocity has mean
n0 + amp sin / Q.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O


def test_uniform_init_is_poisson():
    lat = O.Lattice(O.D2Q5, 96, 64, n0=10.0, seed=3)
    s = lat.init().astype(np.int64).ravel()
    kmax = 30
    obs = np.bincount(np.minimum(s, kmax), minlength=kmax + 1).astype(float)
    pmf = stats.poisson.pmf(np.arange(kmax), 10.0)
    exp = np.append(pmf, 1 - pmf.sum()) * s.size
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    stat = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(stat, len(o) - 1) > 1e-4


@pytest.mark.parametrize("weighted", [0, 1])
def test_sine_profile_means(weighted):
    L, rows = 256, 400
    n0, amp = 30.0, 10.0 if not weighted else 90.0
    lat = O.Lattice(O.D2Q5, L, rows, n0=n0, amp=amp, mode_mx=1, init_weighted=weighted, seed=1)
    s = lat.init().astype(np.float64)
    x = np.arange(L)
    rho = 5 * n0 + amp * np.sin(2 * np.pi * x / L)
    lam = np.array([[lat.init_lambda(int(i), 0, v) for i in x] for v in range(5)])
    assert np.allclose(lam.sum(axis=0), rho, rtol=1e-12)
    if weighted:
        assert np.allclose(lam[0], rho / 3.0, rtol=1e-12)       # w_0 = 1 - 2 theta = 1/3
        assert np.allclose(lam[1:], rho / 6.0, rtol=1e-12)      # w_axis = theta / 2 = 1/6
    else:
        assert np.allclose(lam, (n0 + amp * np.sin(2 * np.pi * x / L) / 5)[None, :], rtol=1e-12)
    colmean = s.mean(axis=1)                                    # (5, L) over rows
    z = (colmean - lam) / np.sqrt(lam / rows)
    assert np.abs(z).max() < 5


def test_init_deterministic_and_replica_keyed():
    a = O.Lattice(O.D1Q3, 500, n0=20.0, seed=8, replica=0).init()
    b = O.Lattice(O.D1Q3, 500, n0=20.0, seed=8, replica=0).init()
    c = O.Lattice(O.D1Q3, 500, n0=20.0, seed=8, replica=1).init()
    d = O.Lattice(O.D1Q3, 500, n0=20.0, seed=9, replica=0).init()
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c) and not np.array_equal(a, d)


def test_init_window_matches_full():
    lat = O.Lattice(O.D2Q5, 40, 30, n0=7.0, amp=5.0, mode_my=2, seed=5)
    full = lat.init()
    win = lat.init_region(35, 27, 10, 6)
    xs = [(35 + i) % 40 for i in range(10)]
    ys = [(27 + j) % 30 for j in range(6)]
    assert np.array_equal(win, full[:, ys][:, :, xs])


def test_negative_mean_rejected():
    lat = O.Lattice(O.D1Q3, 64, n0=1.0, amp=10.0, mode_mx=1, seed=1)
    with pytest.raises(ValueError):
        lat.init()
