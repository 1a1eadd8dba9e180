"""Lattice Boltzmann comparator (ilg_lb_*) against the MRT oracle of Sec. IV, and
the lattice gas's replica mean against it (the Boltzmann average of Sec. IV).

Tolerances (double precision): the device relaxes a node with at most three
rounded operations per output and streams without arithmetic; the oracle takes
a different order (full moment matrix).  Both are contractions of a linear
stable map, so rounding differences add up at most linearly: after T steps the
states agree to |gpu - oracle| <= 1e-15 * (T + 10) * max|f(0)| * 8 per entry.
Mass to 1e-13 relative; projections to 1e-13 of sum |C - M/L| + 1e-9 absolute."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lb as OL
from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


def state_tol(f0, T):
    return 8e-15 * (T + 10) * float(np.abs(f0).max())


CASES = [
    dict(lattice=1, Lx=1000, n0=30.0, amp=10.0, mode_mx=1, init_weighted=0, omega_eff=1.5),
    dict(lattice=1, Lx=257, n0=100.0 / 3.0, amp=100.0, mode_mx=3, init_weighted=1, omega_eff=0.7, theta=0.4),
    dict(lattice=2, Lx=100, Ly=70, n0=50.0, amp=20.0, mode_mx=1, init_weighted=0, omega_eff=1.9),
    dict(lattice=2, Lx=37, Ly=29, n0=7.5, amp=6.0, mode_my=-3, init_weighted=1, omega_eff=1.0, theta=0.25),
    dict(lattice=2, Lx=300, Ly=3, n0=10.0, amp=0.0, omega_eff=0.4),
]


def lb_pair(B, cfg):
    oj, om = OL.rates_from_omega_eff(cfg["omega_eff"])
    kw = {k: v for k, v in cfg.items() if k != "omega_eff"}
    gpu = B.LB(omega_j=oj, omega=om, **kw)
    ora = OL.LB(cfg["lattice"], cfg["Lx"], cfg.get("Ly", 1), theta=cfg.get("theta", 1 / 3), omega_j=oj, omega=om)
    init = {k: cfg.get(k, d) for k, d in (("n0", 10.0), ("amp", 0.0), ("mode_mx", 0), ("mode_my", 0),
                                          ("init_weighted", 0))}
    return gpu, ora, init


@pytest.mark.parametrize("cfg", CASES)
def test_init_is_the_poisson_mean(B, cfg):
    gpu, ora, init = lb_pair(B, cfg)
    with gpu:
        gpu.init()
        f, t = gpu.get_state()
    assert t == 0 and np.array_equal(f, ora.init_mean(**init))


@pytest.mark.parametrize("cfg", CASES)
def test_steps_match_oracle(B, cfg):
    gpu, ora, init = lb_pair(B, cfg)
    T = 40
    with gpu:
        gpu.init()
        gpu.step(T)
        f, t = gpu.get_state()
    f0 = ora.init_mean(**init)
    ref = ora.run(f0, T)
    assert t == T
    assert np.abs(f - ref).max() <= state_tol(f0, T)


@pytest.mark.parametrize("omega_j,omega", [(0.0, 0.0), (2.0, 0.0), (1.0, 1.0), (1.7, 0.6), (0.3, 1.9)])
def test_rates_and_random_state(B, omega_j, omega):
    """Free streaming, pure flip, full relaxation and independent rates from a
    random state set from the host (odd extents, several blocks and a ragged tail)."""
    Lx, Ly, T = 133, 41, 25
    f0 = np.random.default_rng(4).uniform(0.0, 40.0, size=(5, Ly, Lx))
    ora = OL.LB(2, Lx, Ly, omega_j=omega_j, omega=omega)
    with B.LB(2, Lx, Ly, omega_j=omega_j, omega=omega) as gpu:
        gpu.set_state(f0, 5)
        gpu.step(T)
        f, t = gpu.get_state()
    assert t == 5 + T
    assert np.abs(f - ora.run(f0, T)).max() <= state_tol(f0, T)


@pytest.mark.parametrize("cfg", CASES)
def test_observables_match_oracle(B, cfg):
    gpu, ora, init = lb_pair(B, cfg)
    modes = [(1, 0), (2, 0), (-3, 0)] + ([(0, 1), (0, 3)] if cfg["lattice"] == 2 else [])
    with gpu:
        gpu.init()
        gpu.step(15)
        f, _ = gpu.get_state()
        obs = gpu.observables(modes)
    M, res = ora.observables(f, modes)    # the oracle projects the device's own state
    assert abs(obs["mass"] - M) <= 1e-13 * M
    N = f.sum(axis=0)
    for j, (mx, my) in enumerate(modes):
        C = N.sum(axis=0) if my == 0 else N.sum(axis=1)
        scale = float(np.abs(C - M / len(C)).sum())
        tol = 1e-13 * scale + 1e-9
        assert abs(obs["re"][j] - res[j][0]) <= tol, (j, obs["re"][j], res[j][0])
        assert abs(obs["im"][j] - res[j][1]) <= tol
        assert abs(obs["amp"][j] - res[j][2]) <= tol / (f.shape[1] * f.shape[2] / 2)


def test_errors(B):
    with pytest.raises(B.IlgError):
        B.LB(1, 2)
    with pytest.raises(B.IlgError):
        B.LB(1, 64, omega_j=2.5)
    with B.LB(2, 16, 16) as lb:
        with pytest.raises(B.IlgError) as e:
            lb.step(1)
        assert e.value.status == B.ILG_E_STATE
        lb.init()
        with pytest.raises(B.IlgError):
            lb.observables([(1, 1)])
        with pytest.raises(B.IlgError):
            lb.set_state(np.zeros(7))


def test_full_size_workload_y_invariant(B):
    """16384^2 comparator workload in the benchmark's launch: the initial state
    depends on x only, so every row stays equal and equals the oracle run on a
    16384 x 3 lattice; mass conserved."""
    cfg = dict(inputs.LB_D2Q5)
    T = 50
    oj, om = OL.rates_from_omega_eff(cfg["omega_eff"])
    kw = {k: v for k, v in cfg.items() if k not in ("omega_eff", "steps")}
    with B.LB(omega_j=oj, omega=om, **kw) as gpu:
        gpu.init()
        M0 = gpu.observables()["mass"]
        gpu.step(T)
        obs = gpu.observables([(1, 0)])
        f, _ = gpu.get_state()
    assert abs(obs["mass"] - M0) <= 1e-12 * M0
    ora = OL.LB(2, cfg["Lx"], 3, omega_j=oj, omega=om)
    small = ora.init_mean(n0=cfg["n0"], amp=cfg["amp"], mode_mx=cfg["mode_mx"], init_weighted=cfg["init_weighted"])
    ref = ora.run(small, T)
    tol = state_tol(small, T)
    for y in (0, 1, 8191, 16383):
        assert np.abs(f[:, y, :] - ref[:, 0, :]).max() <= tol, y


@pytest.mark.parametrize("sampler", [0, 1])
def test_gas_replica_mean_is_lattice_boltzmann(B, sampler):
    """Sec. IV: the ensemble mean of the gas (either sampler) is the lattice Boltzmann
    solution.  From a Poisson start the gas stays product-Poisson with means f, so
    the mean of R replicas has variance f / R in every entry: chi-square over all
    entries."""
    stats = pytest.importorskip("scipy.stats")
    L, T, R = 96, 30, 400
    base = dict(lattice=1, Lx=L, n0=20.0, amp=30.0, mode_mx=2, init_weighted=1, omega_eff=1.6, seed=23,
                sampler=sampler)
    reps = [dict(base, replica=r) for r in range(R)]
    with B.Batch(reps) as bat:
        bat.init()
        bat.run(T)
        acc = np.zeros((3, 1, L))
        for r in range(R):
            acc += bat.get_state(r)[0]
    mean = acc / R
    oj, om = B.lb_rates(base["omega_eff"])
    with B.LB(1, L, n0=20.0, amp=30.0, mode_mx=2, init_weighted=1, omega_j=oj, omega=om) as lb:
        lb.init()
        lb.step(T)
        f, _ = lb.get_state()
    chi2 = float((((mean - f) ** 2) / (f / R)).sum())
    dof = f.size
    assert stats.chi2.ppf(1e-6, dof) < chi2 < stats.chi2.ppf(1 - 1e-6, dof), chi2


@pytest.mark.parametrize("lattice,Lx,Ly", [(1, 3, 1), (2, 3, 3), (3, 3, 3), (3, 4, 7)])
def test_smallest_lattices(B, lattice, Lx, Ly):
    """Lattices of three nodes per side (neighbours coincide after wrapping) and a mode
    at L/2 (its sine vanishes at every node)."""
    f0 = np.random.default_rng(lattice + Lx).uniform(0.0, 20.0, size=(B.NUM_VEL[lattice], Ly if lattice != 1 else 1, Lx))
    ora = OL.LB(lattice, Lx, Ly, omega_j=1.6, omega=0.4)
    with B.LB(lattice, Lx, Ly, omega_j=1.6, omega=0.4) as gpu:
        gpu.set_state(f0)
        gpu.step(11)
        f, _ = gpu.get_state()
        modes = [(1, 0)] + ([(2, 0)] if Lx % 2 == 0 else [])
        obs = gpu.observables(modes)
    ref = ora.run(f0, 11)
    assert np.abs(f - ref).max() <= 8e-15 * 21 * np.abs(f0).max()
    M, res = ora.observables(f, modes)
    assert abs(obs["mass"] - M) <= 1e-13 * M
    for j in range(len(modes)):
        assert abs(obs["re"][j] - res[j][0]) <= 1e-12 * M and abs(obs["im"][j] - res[j][1]) <= 1e-12 * M
