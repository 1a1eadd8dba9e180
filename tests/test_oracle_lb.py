"""Pins of the MRT lattice Boltzmann oracle (``oracle/lb.py``) against what the
paper and the mathematics fix, not against its own formula.

* Sec. IV: the transform matrix is orthonormal under the weights, both ways.
* Sec. IV, Eq. momentspaceOm: the collision keeps rho, multiplies the current by
  1 - omega^j and the second moments by 1 - omega (moments computed from the
  velocities, not from the matrix).
* Sec. IV, first equation: with omega^j = 2 - omega* the collision equals the flip
  followed by relaxation with omega* towards f^0 (written out per velocity).
* omega^j = omega = 1: the density performs the lattice random walk, rho(t) is the
  t-fold convolution of rho(0) with the weights (brute force).
* omega^j = omega = 0: free streaming; omega^j = 2, omega = 0: period two (Sec. V).
* Sec. IV: a long sine wave decays at the rate D k^2, D = theta (1/omega^j - 1/2).
* Sec. IV: the lattice Boltzmann state is the ensemble mean of the lattice gas;
  since the gas stays product-Poisson from a Poisson start, the replica mean of
  every occupation is within its Poisson error of f (chi-square over all entries).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lb as L


@pytest.mark.parametrize("lattice,theta", [(O.D1Q3, 1 / 3), (O.D1Q3, 0.45), (O.D2Q5, 1 / 3), (O.D2Q5, 0.2),
                                           (O.D2Q9, 1 / 3), (O.D2Q9, 0.6)])
def test_basis_orthonormal_both_ways(lattice, theta):
    m, odd = L.basis(lattice, theta)
    w = np.array(O.weights(lattice, theta))
    Q = len(w)
    assert np.allclose(m @ np.diag(w) @ m.T, np.eye(Q), atol=1e-14)
    assert np.allclose(m.T @ m * w[None, :], np.eye(Q), atol=1e-14)
    v = L.velocities(lattice)
    opp = {O.D1Q3: [0, 2, 1], O.D2Q5: [0, 2, 1, 4, 3], O.D2Q9: [0, 2, 1, 4, 3, 6, 5, 8, 7]}[lattice]
    for a in range(Q):   # odd moments change sign under v -> -v, even ones do not
        assert np.allclose(m[a, opp], -m[a] if odd[a] else m[a])
    assert odd.sum() == {O.D1Q3: 1, O.D2Q5: 2, O.D2Q9: 4}[lattice]


@pytest.mark.parametrize("lattice,omega_j,omega", [(O.D1Q3, 1.6, 0.4), (O.D1Q3, 0.3, 1.7),
                                                   (O.D2Q5, 1.9, 0.1), (O.D2Q5, 0.8, 1.2),
                                                   (O.D2Q9, 1.7, 0.5), (O.D2Q9, 0.4, 1.3)])
def test_moment_space_collision(lattice, omega_j, omega):
    theta = 0.3
    lb = L.LB(lattice, 5, 4, theta=theta, omega_j=omega_j, omega=omega)
    rng = np.random.default_rng(3)
    f = rng.uniform(0.5, 30.0, size=lb.shape)
    g = lb.collide(f)
    v = L.velocities(lattice).astype(float)
    vv = (v * v).sum(axis=1)
    rho, rho2 = f.sum(0), g.sum(0)
    assert np.allclose(rho2, rho, rtol=1e-14)
    for d in range(v.shape[1]):
        j = np.einsum("i,iyx->yx", v[:, d], f)
        assert np.allclose(np.einsum("i,iyx->yx", v[:, d], g), (1 - omega_j) * j, atol=1e-12)
    # second moments about their equilibrium values
    seconds = [vv - v.shape[1] * theta]
    if lattice != O.D1Q3:
        seconds.append(v[:, 0] ** 2 - v[:, 1] ** 2)
    if lattice == O.D2Q9:
        seconds.append(v[:, 0] * v[:, 1])
    for s in seconds:
        pi = np.einsum("i,iyx->yx", s, f)
        assert np.allclose(np.einsum("i,iyx->yx", s, g), (1 - omega) * pi, atol=1e-11)


@pytest.mark.parametrize("lattice,omega_eff", [(O.D1Q3, 1.5), (O.D1Q3, 0.6), (O.D2Q5, 1.8), (O.D2Q5, 1.0),
                                               (O.D2Q9, 1.4), (O.D2Q9, 0.7)])
def test_collision_is_flip_plus_relaxation(lattice, omega_eff):
    oj, om = L.rates_from_omega_eff(omega_eff)
    lb = L.LB(lattice, 6, 3, omega_j=oj, omega=om)
    rng = np.random.default_rng(5)
    f = rng.uniform(0.0, 50.0, size=lb.shape)
    flip, ostar = O.split_omega(omega_eff)
    opp = {O.D1Q3: [0, 2, 1], O.D2Q5: [0, 2, 1, 4, 3], O.D2Q9: [0, 2, 1, 4, 3, 6, 5, 8, 7]}[lattice]
    F = f[opp] if flip else f
    w = np.array(O.weights(lattice, 1 / 3))
    expect = F + ostar * (w[:, None, None] * F.sum(0)[None] - F)
    assert np.allclose(lb.collide(f), expect, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("lattice,Lx,Ly", [(O.D1Q3, 23, 1), (O.D2Q5, 11, 9), (O.D2Q9, 9, 8)])
def test_full_relaxation_is_random_walk(lattice, Lx, Ly):
    lb = L.LB(lattice, Lx, Ly, theta=0.3, omega_j=1.0, omega=1.0)
    rng = np.random.default_rng(8)
    f = rng.uniform(0.0, 10.0, size=lb.shape)
    rho = f.sum(0)
    w = O.weights(lattice, 0.3)
    v = L.velocities(lattice)
    for _ in range(6):
        f = lb.step(f)
        nxt = np.zeros_like(rho)
        for y in range(lb.Ly):          # brute-force convolution with the weights
            for x in range(lb.Lx):
                for i in range(lb.Q):
                    dy = int(v[i, 1]) if lattice != O.D1Q3 else 0
                    nxt[(y + dy) % lb.Ly, (x + int(v[i, 0])) % lb.Lx] += w[i] * rho[y, x]
        rho = nxt
        assert np.allclose(f.sum(0), rho, rtol=1e-13)


@pytest.mark.parametrize("lattice", [O.D1Q3, O.D2Q5, O.D2Q9])
def test_streaming_and_period_two(lattice):
    lb0 = L.LB(lattice, 13, 7, omega_j=0.0, omega=0.0)
    rng = np.random.default_rng(9)
    f = rng.uniform(0.0, 10.0, size=lb0.shape)
    g = lb0.run(f, 5)
    v = L.velocities(lattice)
    for i in range(lb0.Q):
        dy = int(v[i, 1]) if lattice != O.D1Q3 else 0
        assert np.allclose(g[i], np.roll(np.roll(f[i], 5 * int(v[i, 0]), axis=1), 5 * dy, axis=0), rtol=1e-13)
    lb2 = L.LB(lattice, 13, 7, omega_j=2.0, omega=0.0)
    f1 = lb2.step(f)
    assert not np.allclose(f1, f)
    assert np.allclose(lb2.step(f1), f, rtol=1e-14)


@pytest.mark.parametrize("lattice,omega_eff", [(O.D1Q3, 1.5), (O.D1Q3, 0.8), (O.D1Q3, 1.9), (O.D2Q5, 1.3),
                                               (O.D2Q9, 1.6)])
def test_mass_conserved(lattice, omega_eff):
    oj, om = L.rates_from_omega_eff(omega_eff)
    lb = L.LB(lattice, 29, 8, omega_j=oj, omega=om)
    f = np.random.default_rng(1).uniform(0.0, 100.0, size=lb.shape)
    M0 = math.fsum(f.ravel())
    g = lb.run(f, 50)
    assert abs(math.fsum(g.ravel()) - M0) <= 1e-12 * M0


@pytest.mark.parametrize("omega_j", [0.5, 1.0, 1.5, 1.9])
def test_long_wave_decay_rate(omega_j):
    """Sine wave of wavelength 320 (Sec. V) on a D1Q3 ring: after the non-hydrodynamic
    moments have died out, ln A decreases by D k^2 per step, D = theta (1/omega^j - 1/2)."""
    Lx, theta = 320, 1 / 3
    lb = L.LB(O.D1Q3, Lx, theta=theta, omega_j=omega_j, omega=2.0 - omega_j if omega_j > 1 else omega_j)
    x = np.arange(Lx)
    w = np.array(O.weights(O.D1Q3, theta))
    f = w[:, None] * (30.0 * (1.0 + np.sin(2 * np.pi * x / Lx)))[None, None, :]
    f = lb.run(f, 400)
    a0 = lb.observables(f, [(1, 0)])[1][0][1]
    f = lb.run(f, 400)
    a1 = lb.observables(f, [(1, 0)])[1][0][1]
    rate = -math.log(a1 / a0) / 400
    k = 2 * math.pi / Lx
    D = theta * (1 / omega_j - 0.5)
    assert abs(rate / (D * k * k) - 1) < 1e-3


@pytest.mark.parametrize("sampler", [0, 1])
def test_lattice_gas_mean_is_lattice_boltzmann(sampler):
    """Replica mean of the integer lattice gas (oracle, either sampler) after a few
    steps from a Poisson start against the lattice Boltzmann state from the Poisson
    means."""
    cfg = dict(n0=12.0, amp=9.0, mode_mx=1, init_weighted=1, omega_eff=1.6, seed=17, sampler=sampler)
    Lx, T, R = 16, 6, 600
    oj, om = L.rates_from_omega_eff(cfg["omega_eff"])
    lb = L.LB(O.D1Q3, Lx, omega_j=oj, omega=om)
    f = lb.run(lb.init_mean(**{k: v for k, v in cfg.items() if k in ("n0", "amp", "mode_mx", "init_weighted")}), T)
    acc = np.zeros(lb.shape)
    for r in range(R):
        lat = O.Lattice(O.D1Q3, Lx, replica=r, **cfg)
        acc += lat.run(lat.init(), 0, T)
    mean = acc / R
    chi2 = float((((mean - f) ** 2) / (f / R)).sum())
    # chi-square with 48 degrees of freedom: outside [14, 110] has probability < 1e-6
    assert 14 < chi2 < 110, chi2


def test_ensemble_prediction_against_gas_replicas():
    """The exact ensemble statistics (product-Poisson propagation through the lattice
    Boltzmann map) against R replicas of the integer oracle: means, variances and the
    connected correlation with t = 0 of the complex mode amplitude, each within six
    standard errors."""
    cfg = dict(n0=15.0, amp=12.0, mode_mx=1, init_weighted=1, omega_eff=1.7, seed=29)
    Lr, T, R, mode = 12, 8, 2500, 1
    oj, om = L.rates_from_omega_eff(cfg["omega_eff"])
    lb = L.LB(O.D1Q3, Lr, omega_j=oj, omega=om)
    f0 = lb.init_mean(n0=15.0, amp=12.0, mode_mx=1, init_weighted=1)
    pred = L.ensemble_prediction(lb, f0, mode, T)
    lat = O.Lattice(O.D1Q3, Lr, **cfg)
    x = np.arange(Lr)
    cs = np.cos(2 * np.pi * ((mode * x) % Lr) / Lr)
    sn = np.sin(2 * np.pi * ((mode * x) % Lr) / Lr)
    rec = np.zeros((R, T + 1), dtype=complex)
    for r in range(R):
        lat.replica = r
        s = lat.init()
        for t in range(T + 1):
            N = s.sum(axis=0)[0].astype(float)
            rec[r, t] = (cs * N).sum() + 1j * (sn * N).sum()
            if t < T:
                s = lat.step(s, t)
    m = rec.mean(axis=0)
    d = rec - m[None, :]
    var_re = (d.real ** 2).sum(axis=0) / (R - 1)
    var_im = (d.imag ** 2).sum(axis=0) / (R - 1)
    cov = (d * np.conj(d[:, :1])).sum(axis=0) / (R - 1)
    for t in range(T + 1):
        assert abs(m[t].real - pred["mean_re"][t]) < 6 * math.sqrt(pred["var_re"][t] / R)
        assert abs(m[t].imag - pred["mean_im"][t]) < 6 * math.sqrt(pred["var_im"][t] / R)
        assert abs(var_re[t] / pred["var_re"][t] - 1) < 6 * math.sqrt(2 / R) + 0.02
        assert abs(var_im[t] / pred["var_im"][t] - 1) < 6 * math.sqrt(2 / R) + 0.02
        tot0 = pred["var_re"][0] + pred["var_im"][0]
        tot = pred["var_re"][t] + pred["var_im"][t]
        se = math.sqrt(tot * tot0 / R)
        assert abs(cov[t].real - pred["cov_re"][t]) < 6 * se, t
        assert abs(cov[t].imag - pred["cov_im"][t]) < 6 * se, t
    # the correlation must actually decay (omega^j = 1.7: D > 0)
    assert pred["cov_re"][T] < 0.97 * pred["cov_re"][0]


@pytest.mark.parametrize("sampler", [0, 1])
def test_d2q9_gas_mean_is_lattice_boltzmann(sampler):
    """D2Q9: replica mean of the integer oracle against the lattice Boltzmann state."""
    stats = pytest.importorskip("scipy.stats")
    cfg = dict(n0=8.0, amp=20.0, mode_mx=1, init_weighted=1, omega_eff=1.5, seed=19, sampler=sampler)
    Lx, Ly, T, R = 6, 5, 4, 300
    oj, om = L.rates_from_omega_eff(cfg["omega_eff"])
    lb = L.LB(O.D2Q9, Lx, Ly, omega_j=oj, omega=om)
    f = lb.run(lb.init_mean(n0=8.0, amp=20.0, mode_mx=1, init_weighted=1), T)
    lat = O.Lattice(O.D2Q9, Lx, Ly, **cfg)
    acc = np.zeros(lb.shape)
    for r in range(R):
        lat.replica = r
        acc += lat.run(lat.init(), 0, T)
    mean = acc / R
    chi2 = float((((mean - f) ** 2) / (f / R)).sum())
    dof = f.size
    assert stats.chi2.ppf(1e-6, dof) < chi2 < stats.chi2.ppf(1 - 1e-6, dof), chi2
