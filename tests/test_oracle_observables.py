"""Pins of the oracle's observables (Sec. V) and of its light-cone windows, each
against something other than the oracle's own formula:

* the mass and the column / row sums against numpy sums of the state;
* the projections (re, im) against numpy's FFT of D(x) = L C(x) - M (the sign of
  the phase, the normaliser and the mode index), against the closed form of a
  single spike (re + i im = b e^{+2 pi i m x1 / L}) and of a uniform state (zero);
* A^LG against the paper's formula sum_x sin(2 pi m x / L) N(x) / sum_x sin^2(...)
  summed directly, and S(k) against |FFT|^2 / (Lx Ly);
* Lattice.window against the same window cropped from a full periodic run.
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_01380_gb300 import inputs


def fft_projection(sums, M, m):
    """(re, im) as the library defines them, from numpy's FFT:
    fft(D)[m] = sum_x D(x) e^{-2 pi i m x / L} = sum D cos - i sum D sin."""
    L = len(sums)
    D = L * sums.astype(np.float64) - M
    F = np.fft.fft(D)[m % L]
    return F.real / L, -F.imag / L


@pytest.mark.parametrize("lattice,Lx,Ly", [(1, 256, 1), (1, 97, 1), (2, 64, 40), (2, 33, 18), (3, 24, 15)])
def test_sums_match_numpy(lattice, Lx, Ly):
    Q = O.num_vel(lattice)
    s = inputs.random_state(Q, Ly, Lx, 30.0, seed=Lx * Ly, hot=3, hot_value=60000)
    ref = O.Lattice(lattice, Lx, Ly)
    M, col, row = ref.sums(s)
    N = s.astype(np.int64).sum(axis=0)
    assert M == int(N.sum())
    assert np.array_equal(col, N.sum(axis=0)) and np.array_equal(row, N.sum(axis=1))


@pytest.mark.parametrize("lattice,Lx,Ly,modes", [
    (1, 256, 1, [(1, 0), (2, 0), (5, 0), (127, 0), (255, 0), (-3, 0)]),
    (1, 97, 1, [(1, 0), (48, 0), (96, 0)]),
    (2, 64, 40, [(1, 0), (7, 0), (0, 1), (0, 13), (0, 39)]),
    (3, 30, 21, [(2, 0), (0, 5)]),
])
def test_projections_match_fft(lattice, Lx, Ly, modes):
    """Every mode of a random state: re, im, A^LG and S(k) against numpy's FFT of D."""
    Q = O.num_vel(lattice)
    s = inputs.random_state(Q, Ly, Lx, 40.0, seed=7 + Lx, hot=2, hot_value=900)
    ref = O.Lattice(lattice, Lx, Ly)
    M, col, row, res = ref.observables(s, modes)
    K = Lx * Ly
    for (mx, my), r in zip(modes, res):
        sums, m = (col, mx) if my == 0 else (row, my)
        re, im = fft_projection(sums, M, m)
        tol = 1e-12 * r["scale"] + 1e-9
        assert abs(r["re"] - re) <= tol and abs(r["im"] - im) <= tol, (mx, my, r, re, im)
        assert abs(r["amp"] - im / (K / 2.0)) <= tol / (K / 2.0)
        assert abs(r["Sk"] - (re * re + im * im) / K) <= 1e-10 * (re * re + im * im + 1.0) / K


@pytest.mark.parametrize("L,m,x1,b", [(256, 1, 0, 5), (256, 1, 64, 7), (256, 3, 10, 1000), (320, 1, 80, 3),
                                      (97, 5, 31, 12), (12, 5, 7, 65535)])
def test_single_spike_closed_form(L, m, x1, b):
    """C(x) = c + b [x = x1]: D(x) = L b [x = x1] - b, so re + i im = b e^{2 pi i m x1 / L}
    (the uniform part cancels for m not a multiple of L), and S(k) = b^2 / L."""
    c = 3
    s = np.zeros((3, 1, L), dtype=np.uint16)
    s[0, 0, :] = c
    s[1, 0, x1] = b
    ref = O.Lattice(1, L)
    M, col, row, res = ref.observables(s, [(m, 0)])
    r = res[0]
    phase = 2.0 * np.pi * ((m * x1) % L) / L
    assert abs(r["re"] - b * np.cos(phase)) <= 1e-12 * b * 2
    assert abs(r["im"] - b * np.sin(phase)) <= 1e-12 * b * 2
    assert abs(r["Sk"] - b * b / L) <= 1e-12 * b * b / L


def test_uniform_state_projects_to_zero():
    """Equal column sums: D = 0 everywhere, every projection exactly zero."""
    s = np.full((5, 8, 32), 11, dtype=np.uint16)
    ref = O.Lattice(2, 32, 8)
    _, _, _, res = ref.observables(s, [(1, 0), (3, 0), (0, 1), (0, 2)])
    for r in res:
        assert r["re"] == 0.0 and r["im"] == 0.0 and r["amp"] == 0.0 and r["Sk"] == 0.0


@pytest.mark.parametrize("L,m,c,a", [(320, 1, 100, 100.0), (256, 2, 300, 40.0), (97, 3, 50, 20.0)])
def test_amplitude_is_the_papers_formula(L, m, c, a):
    """A^LG of Sec. V, sum_x sin(2 pi m x / L) N(x) / sum_x sin^2(2 pi m x / L), summed
    directly in double precision over a state N(x) = c + round(a sin(2 pi m x / L)) split
    over the velocities; and it recovers a to within the rounding of N."""
    x = np.arange(L)
    sin = np.sin(2.0 * np.pi * m * x / L)
    N = c + np.rint(a * sin).astype(np.int64)
    s = np.zeros((3, 1, L), dtype=np.uint16)
    s[0, 0] = N // 3
    s[1, 0] = N // 3
    s[2, 0] = N - 2 * (N // 3)
    ref = O.Lattice(1, L)
    _, _, _, res = ref.observables(s, [(m, 0)])
    direct = float(np.sum(sin * N) / np.sum(sin * sin))
    assert abs(res[0]["amp"] - direct) <= 1e-10 * a
    # rounding N moves A by at most sum |sin| / 2 / (L / 2) < 0.64
    assert abs(res[0]["amp"] - a) < 0.64


@pytest.mark.parametrize("lattice,Lx,Ly,x0,y0,w,h,t0,steps", [
    (1, 64, 1, 0, 0, 12, 1, 0, 9),        # across the ring's periodic seam
    (1, 50, 1, 45, 0, 9, 1, 5, 7),
    (2, 40, 32, 0, 0, 6, 5, 0, 6),        # the corner: wraps in x and y
    (2, 40, 32, 30, 25, 8, 7, 3, 5),
    (2, 24, 24, 10, 3, 5, 9, 0, 8),
    (3, 20, 18, 17, 0, 6, 6, 0, 5),
])
@pytest.mark.parametrize("omega_eff", [0.6, 1.8])
def test_window_equals_cropped_full_run(lattice, Lx, Ly, x0, y0, w, h, t0, steps, omega_eff):
    """The light-cone window (the parity tests' route at full size) equals the window of
    the full periodic run, from the oracle's own initial state and from a given one."""
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, n0=12.0, amp=5.0, mode_mx=1, omega_eff=omega_eff, seed=21, replica=2)
    ref = O.Lattice(**cfg)
    full0 = ref.init()
    if t0:
        full0 = ref.run(full0, 0, t0)
    full = ref.run(full0, t0, steps)
    ys = (np.arange(y0, y0 + h) % ref.Ly) if lattice != 1 else np.array([0])
    xs = np.arange(x0, x0 + w) % Lx
    want = full[:, ys][:, :, xs]
    if t0 == 0:
        got = ref.window(x0, y0, w, h, steps)
        assert np.array_equal(got, want)
    # from a given initial patch: the (w + 2s) x (h + 2s) neighbourhood of the window
    pad_y = steps if lattice != 1 else 0
    pys = (np.arange(y0 - pad_y, y0 + h + pad_y) % ref.Ly) if lattice != 1 else np.array([0])
    pxs = np.arange(x0 - steps, x0 + w + steps) % Lx
    patch = np.ascontiguousarray(full0[:, pys][:, :, pxs])
    got = ref.window(x0, y0, w, h, t0 + steps, t0=t0, initial=patch)
    assert np.array_equal(got, want)
