"""Pins of the oracle's sampling collision against the law the paper states.

Sec. II: the collision picks particles at random with probability omega and
redistributes each picked particle to velocity j with probability w_j.  Per
particle at velocity i that is the transition matrix
    P_ij = (1 - omega) delta_ij + omega w_j,
so the post-collision occupation is a sum of independent multinomials.  The
tests enumerate that law exactly (rational arithmetic, tiny occupations) and
compare the oracle's sampled histograms to it, check first and second moments
at large occupations (where the sampler splits binomials into chunks and needs
extension words), and check the moment-space picture of Sec. IV: after the
flip and the collision the current j is multiplied by (1 - omega^j) with
omega^j = 2 - omega, and the ghost moment Pi by (1 - omega).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import sympy
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_d1q3.json")


def transition(lat: O.Lattice):
    """P_ij with the quantised probabilities the sampler uses."""
    Q = lat.Q
    om = Fraction(lat.P_omega, 1 << 32)
    w0 = Fraction(lat.P_rest, 1 << 32)
    if Q == 9:
        pa = Fraction(lat.P_axis, 1 << 32)
        w = [w0] + [(1 - w0) * pa / 4] * 4 + [(1 - w0) * (1 - pa) / 4] * 4
    else:
        w = [w0] + [(1 - w0) / (Q - 1)] * (Q - 1)
    return [[(1 - om) * (1 if i == j else 0) + om * w[j] for j in range(Q)] for i in range(Q)]


def exact_law(lat: O.Lattice, m):
    P = transition(lat)
    dist = {tuple([0] * lat.Q): Fraction(1)}
    for i, mi in enumerate(m):
        for _ in range(mi):
            nxt = {}
            for out, pr in dist.items():
                for j in range(lat.Q):
                    if P[i][j] == 0:
                        continue
                    o = list(out)
                    o[j] += 1
                    o = tuple(o)
                    nxt[o] = nxt.get(o, 0) + pr * P[i][j]
            dist = nxt
    return dist


def chi2_pvalue(samples: np.ndarray, law: dict) -> float:
    n = len(samples)
    keys = [tuple(int(v) for v in row) for row in samples]
    counts = {}
    for k in keys:
        counts[k] = counts.get(k, 0) + 1
    assert set(counts) <= set(law), "sampled an outcome of probability zero"
    obs, exp = [], []
    rest_o, rest_e = 0, 0.0
    for k, p in law.items():
        e = float(p) * n
        if e < 5:
            rest_o += counts.get(k, 0)
            rest_e += e
        else:
            obs.append(counts.get(k, 0))
            exp.append(e)
    if rest_e > 0:
        obs.append(rest_o)
        exp.append(rest_e)
    obs, exp = np.array(obs, float), np.array(exp)
    stat = float(((obs - exp) ** 2 / exp).sum())
    return float(stats.chi2.sf(stat, len(obs) - 1))


CASES = [
    (O.D1Q3, (2, 3, 1), 0.3, 1.0 / 3.0),
    (O.D1Q3, (0, 4, 0), 0.75, 1.0 / 3.0),
    (O.D1Q3, (5, 0, 0), 1.0, 1.0 / 3.0),
    (O.D1Q3, (0, 0, 5), 1.0, 1.0 / 3.0),
    (O.D1Q3, (1, 2, 2), 0.5, 0.6),
    (O.D2Q5, (1, 2, 0, 1, 2), 0.45, 1.0 / 3.0),
    (O.D2Q5, (3, 0, 0, 0, 0), 1.0, 1.0 / 3.0),
    (O.D2Q5, (0, 0, 1, 1, 1), 1.0, 1.0 / 3.0),
    (O.D2Q5, (2, 1, 1, 1, 1), 0.6, 0.4),
    (O.D2Q5, (0, 3, 0, 0, 2), 0.05, 1.0 / 3.0),
    (O.D2Q9, (1, 1, 0, 0, 0, 1, 0, 0, 1), 0.5, 1.0 / 3.0),
    (O.D2Q9, (0, 0, 0, 0, 0, 2, 0, 0, 0), 1.0, 1.0 / 3.0),
    (O.D2Q9, (2, 0, 1, 0, 0, 0, 0, 1, 0), 0.7, 0.45),
]


@pytest.mark.parametrize("lattice,m,omega,theta", CASES)
def test_collision_law_exact(lattice, m, omega, theta):
    lat = O.Lattice(lattice, 16, 16, omega_eff=omega, theta=theta, seed=11 + sum(m))
    law = exact_law(lat, m)
    assert abs(sum(law.values()) - 1) == 0
    out = lat.collide_many(m, t=5, node0=0, count=200_000)
    assert np.all(out.sum(axis=1) == sum(m))  # exact mass conservation per node
    assert chi2_pvalue(out, law) > 1e-4


@pytest.mark.parametrize("lattice,m,omega", [
    (O.D2Q9, (120, 70, 0, 45, 200, 5, 66, 90, 1), 0.6),
    (O.D2Q9, (20, 20, 20, 20, 20, 20, 20, 20, 20), 1.0),
    (O.D2Q5, (300, 70, 0, 45, 200), 0.5),
    (O.D2Q5, (40, 40, 40, 40, 40), 0.9),
    (O.D1Q3, (150, 260, 90), 0.8),
    (O.D1Q3, (65, 64, 1), 0.35),
])
def test_collision_moments_large(lattice, m, omega):
    """Chunked binomials (m_i > 64) and more than 32 moving particles."""
    lat = O.Lattice(lattice, 16, 16, omega_eff=omega, seed=5)
    P = np.array([[float(v) for v in row] for row in transition(lat)])
    mm = np.array(m, float)
    mean = mm @ P
    cov = -np.einsum("i,ij,ik->jk", mm, P, P) + np.diag(mm @ P)
    n = 100_000
    out = lat.collide_many(m, t=9, node0=1000, count=n).astype(float)
    assert np.all(out.sum(axis=1) == sum(m))
    z = (out.mean(axis=0) - mean) / np.sqrt(np.diag(cov) / n)
    assert np.all(np.abs(z) < 5), z
    c = np.cov(out.T)
    # sample covariance error ~ sqrt((var_j var_k + cov^2) / n)
    err = np.sqrt((np.outer(np.diag(cov), np.diag(cov)) + cov ** 2) / n)
    assert np.all(np.abs(c - cov) < 6 * err + 1e-9)


def test_moment_space_collision_with_flip():
    """Sec. IV: flip maps (rho, j, Pi) -> (rho, -j, Pi); the collision multiplies
    the non-conserved moments by (1 - omega*); so after flip + collision the mean
    moments are (rho, (1 - omega^j) j, (1 - omega*) Pi) with omega^j = 2 - omega*."""
    g = json.load(open(GOLDEN))
    theta = sympy.Rational(1, 3)
    th = sympy.Symbol("theta")
    M = np.array([[float(sympy.sympify(e).subs(th, theta)) for e in row] for row in g["transform"]])
    # the paper's velocity order is (-1, 0, +1); storage order is (0, +1, -1)
    paper_to_store = [2, 0, 1]
    omega_eff = 1.6
    lat = O.Lattice(O.D1Q3, 16, omega_eff=omega_eff, theta=float(theta), seed=21)
    assert lat.flip == 1
    omega_star = 2.0 - omega_eff
    n_paper = np.array([40.0, 10.0, 25.0])            # n_{-1}, n_0, n_{+1}
    n_store = np.zeros(3)
    for p, s in enumerate(paper_to_store):
        n_store[s] = n_paper[p]
    flipped = n_store[[0, 2, 1]]                      # F_i(n) = n_{-i}
    out = lat.collide_many(flipped.astype(np.uint32), t=3, node0=0, count=200_000).astype(float)
    out_paper = out[:, paper_to_store]
    mom_in = M @ n_paper
    mom_out = out_paper @ M.T
    omega_j = 2.0 - omega_star
    expect = np.array([mom_in[0], (1 - omega_j) * mom_in[1], (1 - omega_star) * mom_in[2]])
    se = mom_out.std(axis=0) / np.sqrt(len(out))
    assert abs(mom_out[:, 0].mean() - expect[0]) < 1e-9   # mass is exact
    for a in (1, 2):
        assert abs(mom_out[:, a].mean() - expect[a]) < 5 * se[a], (a, mom_out[:, a].mean(), expect[a])


def test_paper_transform_is_hermite_orthogonal_with_weights():
    """Sec. IV: sum_i m_i^a w_i m_i^b = delta^ab holds for the paper's D1Q3
    matrix exactly when w_{+-1} = theta/2 and w_0 = 1 - theta (the weights the
    oracle uses), for any theta in (0, 1)."""
    g = json.load(open(GOLDEN))
    th = sympy.Symbol("theta", positive=True)
    M = sympy.Matrix([[sympy.sympify(e, locals={"theta": th}) for e in row] for row in g["transform"]])
    w = sympy.diag(th / 2, 1 - th, th / 2)              # paper order (-1, 0, +1)
    G = sympy.simplify(M * w * M.T)
    for val in (sympy.Rational(1, 3), sympy.Rational(1, 5), sympy.Rational(7, 10)):
        assert sympy.simplify(G.subs(th, val) - sympy.eye(3)) == sympy.zeros(3)
    ow = O.weights(O.D1Q3, 0.25)
    assert ow == [0.75, 0.125, 0.125]
    assert O.weights(O.D2Q5, 1.0 / 3.0)[0] == pytest.approx(1.0 / 3.0)


# ---------------------------------------------------------------- particle sampler
# The plain per-particle form of the same collision: one word per particle against
# integer boundaries.  Its law must be the paper's (Sec. II) to within the 2^-32
# quantisation, so it is compared with the same exact enumeration.

@pytest.mark.parametrize("lattice,omega,theta", [(O.D1Q3, 0.3, 1 / 3), (O.D1Q3, 1.0, 0.6), (O.D2Q5, 0.45, 1 / 3),
                                                 (O.D2Q5, 0.0, 0.4), (O.D2Q5, 1.0, 0.2), (O.D2Q9, 0.3, 1 / 3),
                                                 (O.D2Q9, 1.0, 0.6)])
def test_particle_bounds_realise_the_law(lattice, omega, theta):
    lat = O.Lattice(lattice, 8, 8, omega_eff=omega, theta=theta)
    B = O.particle_bounds(lattice, lat.P_omega, lat.P_rest, lat.P_axis)
    Q = lat.Q
    assert len(B) == Q + 1 and B[-1] == 1 << 32
    assert all(B[k] <= B[k + 1] for k in range(Q))
    w = O.weights(lattice, theta)
    two32 = float(1 << 32)
    assert abs(B[0] / two32 - (1 - omega)) <= 1.5 / two32
    for j in range(Q):
        assert abs((B[j + 1] - B[j]) / two32 - omega * w[j]) <= 3 / two32, j


@pytest.mark.parametrize("lattice,m,omega,theta", CASES)
def test_particle_sampler_law_exact(lattice, m, omega, theta):
    lat = O.Lattice(lattice, 16, 16, omega_eff=omega, theta=theta, seed=23 + sum(m), sampler=1)
    law = exact_law(lat, m)
    out = lat.collide_many(m, t=3, node0=0, count=200_000)
    assert np.all(out.sum(axis=1) == sum(m))
    assert chi2_pvalue(out, law) > 1e-4


@pytest.mark.parametrize("lattice,m,omega", [(O.D2Q5, (300, 70, 0, 45, 200), 0.5), (O.D1Q3, (150, 260, 90), 0.8),
                                             (O.D2Q9, (30, 70, 0, 45, 20, 5, 66, 90, 1), 0.6)])
def test_particle_sampler_moments_large(lattice, m, omega):
    lat = O.Lattice(lattice, 16, 16, omega_eff=omega, seed=6, sampler=1)
    P = np.array([[float(v) for v in row] for row in transition(lat)])
    mm = np.array(m, float)
    mean = mm @ P
    cov = -np.einsum("i,ij,ik->jk", mm, P, P) + np.diag(mm @ P)
    n = 30_000
    out = lat.collide_many(m, t=2, node0=7, count=n).astype(float)
    assert np.all(out.sum(axis=1) == sum(m))
    z = (out.mean(axis=0) - mean) / np.sqrt(np.diag(cov) / n)
    assert np.all(np.abs(z) < 5), z


def test_particle_sampler_special_cases():
    """omega* = 0 keeps every particle (Sec. V: the pure flip); the two samplers differ
    in their bits but not in mass."""
    m = (7, 3, 0, 11, 2)
    keep = O.Lattice(O.D2Q5, 8, 8, omega_eff=2.0, seed=1, sampler=1)
    assert keep.P_omega == 0
    out = keep.collide_many(m, t=0, node0=0, count=50)
    assert np.all(out == np.array(m))
    a = O.Lattice(O.D2Q5, 8, 8, omega_eff=0.7, seed=1, sampler=1).collide_many(m, t=0, node0=0, count=50)
    b = O.Lattice(O.D2Q5, 8, 8, omega_eff=0.7, seed=1, sampler=0).collide_many(m, t=0, node0=0, count=50)
    assert not np.array_equal(a, b)
    assert np.all(a.sum(axis=1) == sum(m)) and np.all(b.sum(axis=1) == sum(m))
