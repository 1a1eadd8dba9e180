"""Pins of the oracle's time step (flip -> collision -> streaming) against what
the paper and the mathematics fix.

* Sec. V: at omega^j = 2 (omega* = 0) the system does not evolve: flip plus
  streaming returns every particle after two steps, bit for bit.
* Sec. II, Eq. 2: mass is conserved exactly, every step.
* Sec. IV: the ensemble mean of the lattice gas follows the lattice Boltzmann
  equation f(x+v, t+1) = F f + omega* (f^0 - F f) (with flip) or
  f + omega (f^0 - f) (without); the mean amplitude of a sine wave is compared
  with that deterministic evolution, and its decay rate with D k^2 for
  D = theta (1/omega^j - 1/2) (Sec. IV) and D = theta (1/omega - 1/2) (Sec. II).
* Fluctuations: binomial thinning, multinomial redistribution, the flip and
  streaming all map independent Poisson occupations to independent Poisson
  occupations, so an equilibrium Poisson state stays product-Poisson: the
  structure factor S(k) equals the mean density for every k != 0 and every
  occupation has variance equal to its mean.
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_01380_gb300 import inputs


@pytest.mark.parametrize("lattice,Lx,Ly", [(O.D1Q3, 37, 1), (O.D2Q5, 19, 13), (O.D2Q9, 11, 9)])
def test_pure_flip_has_period_two(lattice, Lx, Ly):
    lat = O.Lattice(lattice, Lx, Ly, omega_eff=2.0, seed=7)
    assert lat.flip == 1 and lat.P_omega == 0
    s0 = inputs.random_state(lat.Q, lat.Ly, lat.Lx, 12.0, seed=1)
    s1 = lat.step(s0, 0)
    s2 = lat.step(s1, 1)
    assert not np.array_equal(s1, s0)
    assert np.array_equal(s2, s0)
    assert np.array_equal(lat.run(s0, 10, 8), s0)


@pytest.mark.parametrize("lattice,omega", [(O.D1Q3, 0.7), (O.D1Q3, 1.9), (O.D2Q5, 1.0), (O.D2Q5, 1.3),
                                          (O.D2Q9, 0.8), (O.D2Q9, 1.6)])
def test_mass_conserved_every_step(lattice, omega):
    lat = O.Lattice(lattice, 33, 17, omega_eff=omega, seed=9)
    s = inputs.random_state(lat.Q, lat.Ly, lat.Lx, 20.0, seed=2, hot=5, hot_value=700)
    M0 = int(s.astype(np.int64).sum())
    for t in range(40):
        s = lat.step(s, t)
        assert int(s.astype(np.int64).sum()) == M0


def lb_mean(lat: O.Lattice, f: np.ndarray, steps: int) -> list:
    """Deterministic mean dynamics of Sec. IV on a D1Q3 ring, f shape (3, L);
    returns the sine amplitude (mode 1 of the ring's mode) after each step."""
    w = np.array(lat.w)
    om = lat.omega_star
    opp = [0, 2, 1]
    out = []
    for _ in range(steps):
        g = f[opp] if lat.flip else f
        rho = g.sum(axis=0)
        post = g + om * (w[:, None] * rho[None, :] - g)
        f = np.stack([post[0], np.roll(post[1], 1), np.roll(post[2], -1)])
        out.append(f)
    return out


def amplitude(N: np.ndarray, m: int) -> float:
    L = len(N)
    s = np.sin(2 * np.pi * m * np.arange(L) / L)
    return float((s * N).sum() / (L / 2))


@pytest.mark.parametrize("omega_j,steps,check_D", [(0.5, 220, True), (1.5, 1200, True), (1.9, 300, False)])
def test_sine_decay_mean_dynamics_and_diffusion(omega_j, steps, check_D):
    """Long ring of R wavelengths (64 nodes each) stands in for an ensemble of R
    rings: the mode amplitude of wavelength 64 follows the mean dynamics."""
    R, lam = 120, 64
    L = R * lam
    n_ave = 100.0
    theta = 1.0 / 3.0
    lat = O.Lattice(O.D1Q3, L, n0=n_ave / 3.0, amp=n_ave, mode_mx=R, init_weighted=1,
                    omega_eff=omega_j, theta=theta, seed=31)
    s = lat.init()
    x = np.arange(L)
    f0 = np.stack([np.array([lat.init_lambda(int(i), 0, v) for i in x]) for v in range(3)])
    pred = [amplitude(fk.sum(axis=0), R) for fk in lb_mean(lat, f0, steps)]
    sigma = np.sqrt(2 * n_ave / L) * 1.5  # product-Poisson noise of A (with margin for sine weighting)
    meas = []
    for t in range(steps):
        s = lat.step(s, t)
        meas.append(amplitude(s.astype(np.int64).sum(axis=0)[0], R))
    meas = np.array(meas)
    pred = np.array(pred)
    idx = np.linspace(0, steps - 1, 12).astype(int)
    assert np.all(np.abs(meas[idx] - pred[idx]) < 5 * sigma), (meas[idx], pred[idx])
    if check_D:
        D = theta * (1.0 / omega_j - 0.5)
        k = 2 * np.pi / lam
        t = np.arange(1, steps + 1)
        sel = t > steps // 5
        slope = np.polyfit(t[sel], np.log(meas[sel]), 1)[0]
        assert abs(-slope / (D * k * k) - 1) < 0.05, (-slope, D * k * k)


def test_equilibrium_is_product_poisson():
    lat = O.Lattice(O.D2Q5, 64, 64, n0=20.0, init_weighted=1, omega_eff=1.8, seed=41)
    s = lat.run(lat.init(), 0, 30).astype(np.float64)
    lam = np.array([lat.init_lambda(0, 0, v) for v in range(5)])
    for v in range(5):
        x = s[v].ravel()
        assert abs(x.mean() / lam[v] - 1) < 0.02
        assert abs(x.var() / x.mean() - 1) < 0.1
    c = np.corrcoef(s[0].ravel(), s[1].ravel())[0, 1]
    assert abs(c) < 0.08
    N = s.sum(axis=0)
    F = np.fft.fft2(N - N.mean())
    Sk = (np.abs(F) ** 2 / N.size).ravel()[1:]
    rho = lam.sum()
    assert abs(Sk.mean() / rho - 1) < 0.08


@pytest.mark.parametrize("lattice,Lx,Ly", [(O.D1Q3, 23, 1), (O.D2Q5, 11, 7), (O.D2Q9, 10, 7)])
def test_free_streaming_direction(lattice, Lx, Ly):
    """With omega_eff so small that omega* quantises to 0 (and no flip) the step is
    streaming alone, n_i(x + v_i, t + 1) = n_i(x, t) (Sec. II, Eq. ilgeq), with
    v = (0, +1, -1) on D1Q3 and (0, +x, -x, +y, -y) on D2Q5 (y = row index)."""
    lat = O.Lattice(lattice, Lx, Ly, omega_eff=1e-12, seed=3)
    assert lat.P_omega == 0 and lat.flip == 0
    s = inputs.random_state(lat.Q, lat.Ly, lat.Lx, 9.0, seed=4)
    out = lat.step(s, 0)
    shifts = {O.D1Q3: [(0, 0), (0, 1), (0, -1)],
              O.D2Q5: [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0)],
              O.D2Q9: [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0), (1, 1), (-1, -1), (-1, 1), (1, -1)]}[lattice]
    for v, (dy, dx) in enumerate(shifts):
        assert np.array_equal(out[v], np.roll(np.roll(s[v], dy, axis=0), dx, axis=1)), v
