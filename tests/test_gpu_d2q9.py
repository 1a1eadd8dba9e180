"""D2Q9 lattices (ilg_create with ILG_D2Q9, and the comparator) against the oracle:
initial states, states after T steps with both samplers (every flip / omega* regime,
occupations far above the fast path, odd extents and even ones, which take two nodes
per thread), observables, overflow rollback,
the 16384^2 workload through a light-cone window, and the replica mean against the
lattice Boltzmann comparator."""
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


@pytest.mark.parametrize("cfg", [
    dict(Lx=40, Ly=33, n0=10.0, amp=30.0, mode_mx=1, init_weighted=1, seed=2),
    dict(Lx=17, Ly=64, n0=25.0, amp=9.0, mode_my=-2, init_weighted=0, seed=5, replica=9, theta=0.45),
    dict(Lx=96, Ly=5, n0=3.0, seed=7),
])
def test_init_bit_exact(B, cfg):
    cfg = dict(cfg, lattice=3)
    with B.Lattice(**cfg) as lat:
        lat.init()
        got, t = lat.get_state()
    assert t == 0 and np.array_equal(got, O.Lattice(**cfg).init())


STEP_CASES = [
    # Lx, Ly, omega_eff, theta, mean, hot, sampler
    (64, 40, 1.8, 1 / 3, 10.0, 0, 0),
    (37, 29, 0.7, 1 / 3, 12.0, 4, 0),
    (50, 21, 1.0, 0.5, 20.0, 0, 0),      # omega* = 1
    (24, 24, 2.0, 1 / 3, 9.0, 0, 0),     # omega* = 0: pure flip
    (33, 17, 1.4, 0.2, 70.0, 3, 0),      # general path: chunks, extension words
    (31, 19, 1.6, 1 / 3, 8.0, 2, 1),     # particle sampler
    (40, 12, 0.5, 0.6, 15.0, 0, 1),
    # even rows take two nodes per thread: the pair at the row's end wraps to x = 0
    (4, 5, 1.7, 1 / 3, 30.0, 2, 0),
    (6, 3, 0.9, 0.4, 70.0, 1, 0),
    (34, 7, 1.2, 1 / 3, 11.0, 0, 1),
]


@pytest.mark.parametrize("Lx,Ly,omega,theta,mean,hot,sampler", STEP_CASES)
def test_steps_bit_exact(B, Lx, Ly, omega, theta, mean, hot, sampler):
    s0 = inputs.random_state(9, Ly, Lx, mean, seed=Lx * 3 + Ly, hot=hot, hot_value=900)
    cfg = dict(lattice=3, Lx=Lx, Ly=Ly, omega_eff=omega, theta=theta, seed=13, replica=2, sampler=sampler)
    with B.Lattice(**cfg) as lat:
        lat.set_state(s0, 21)
        lat.step(8)
        got, t = lat.get_state()
    assert t == 29 and np.array_equal(got, O.Lattice(**cfg).run(s0, 21, 8))


@pytest.mark.parametrize("kernel", [2, 6, 7])
@pytest.mark.parametrize("Lx,Ly,omega,theta,mean,hot,hot_value", [
    (96, 40, 1.8, 1 / 3, 10.0, 3, 900),   # several tiles per row; nodes for the general collision
    (100, 23, 0.7, 0.45, 5.0, 6, 60),     # ragged last tile; no flip; nodes whose removals pass 63
    (2056, 9, 1.3, 1 / 3, 6.0, 1, 900),   # segments split at row ends across warps
    (8200, 3, 1.6, 0.45, 9.0, 0, 0),      # long rows, few of them
    (4, 5, 1.7, 1 / 3, 12.0, 0, 0),       # one vector per row: both its ends wrap
    (36, 3, 0.9, 0.3, 4.0, 1, 60),        # three rows: every diagonal wraps
])
def test_step_kernels_bit_exact(B, kernel, Lx, Ly, omega, theta, mean, hot, hot_value):
    """The node-parallel D2Q9 step (candidate 2) and the staged warp step with
    4-node vectors in 384 or 256 threads (candidates 6, 7) give the oracle's bits."""
    s0 = inputs.random_state(9, Ly, Lx, mean, seed=Lx + 7 * Ly, hot=hot, hot_value=hot_value)
    # mean removals per node low enough for the lattice to keep its fast-path kernels
    omega_star = 2.0 - omega if omega > 1.0 else omega
    assert omega_star * 9 * s0.mean() <= 40.0
    cfg = dict(lattice=3, Lx=Lx, Ly=Ly, omega_eff=omega, theta=theta, seed=17, replica=3)
    with B.Lattice(**cfg) as lat:
        lat.set_step_kernel(kernel)
        lat.set_state(s0, 5)
        lat.step(7)
        got, t = lat.get_state()
    assert t == 12 and np.array_equal(got, O.Lattice(**cfg).run(s0, 5, 7))


def test_observables_and_overflow(B):
    cfg = dict(lattice=3, Lx=30, Ly=22, n0=12.0, amp=40.0, mode_mx=2, init_weighted=1, omega_eff=1.3, seed=4)
    ref = O.Lattice(**cfg)
    s = ref.run(ref.init(), 0, 5)
    modes = [(1, 0), (2, 0), (0, 1), (0, -3)]
    with B.Lattice(**cfg) as lat:
        lat.init()
        lat.step(5)
        obs = lat.observables(modes, col_sums=True, row_sums=True)
    M, col, row, res = ref.observables(s, modes)
    assert obs["mass"] == M and np.array_equal(obs["col"], col) and np.array_equal(obs["row"], row)
    for j, r in enumerate(res):
        tol = 1e-12 * r["scale"] + 1e-12
        assert abs(obs["re"][j] - r["re"]) <= tol and abs(obs["im"][j] - r["im"]) <= tol
    # overflow: the failing step is rolled back
    s0 = inputs.random_state(9, 10, 10, 3.0, seed=8)
    s0[:, 4, 4] = 30000
    cfg2 = dict(lattice=3, Lx=10, Ly=10, omega_eff=1.0, seed=4)
    ref2 = O.Lattice(**cfg2)
    cur, fail_t = s0.copy(), None
    for t in range(6):
        try:
            cur = ref2.step(cur, t)
        except OverflowError:
            fail_t = t
            break
    assert fail_t is not None
    with B.Lattice(**cfg2) as lat:
        lat.set_state(s0, 0)
        with pytest.raises(B.IlgError) as e:
            lat.step(6)
        assert e.value.status == B.ILG_E_OVERFLOW
        got, t = lat.get_state()
    assert t == fail_t and np.array_equal(got, cur)


def test_unsupported_paths_rejected(B):
    with B.Lattice(lattice=3, Lx=16, Ly=16) as lat:
        with pytest.raises(B.IlgError):
            lat.set_temporal_blocking(2)
    with pytest.raises(B.IlgError):
        B.Batch([dict(lattice=3, Lx=16, Ly=16)])
    with pytest.raises(B.IlgError):
        B.Lattice(lattice=3, Lx=16, Ly=16, theta=1.0)


def test_large_d2q9_light_cone_full_size(B):
    """16384^2 D2Q9 workload in the benchmark's launch: a 10 x 10 window at t = 100
    from the oracle's own initial state of its light cone; plus exact mass."""
    cfg = {k: v for k, v in inputs.LARGE_D2Q9.items() if k != "steps"}
    steps = inputs.LARGE_D2Q9["steps"]
    x0, y0, w = 3, 16384 - 4, 10
    with B.Lattice(**cfg) as lat:
        lat.init()
        m0 = lat.observables()["mass"]
        lat.step(steps)
        obs = lat.observables()
        state = np.empty(lat.shape, np.uint16)
        lat.get_state(state)
    assert obs["mass"] == m0
    win = O.Lattice(**cfg).window(x0, y0, w, w, steps)
    ys = [(y0 + j) % 16384 for j in range(w)]
    assert np.array_equal(state[:, ys][:, :, x0:x0 + w], win)


def test_comparator_d2q9_and_replica_mean(B):
    """The comparator on D2Q9 against the oracle, and the mean of 200 gas replicas
    against it (chi-square over every entry)."""
    stats = pytest.importorskip("scipy.stats")
    Lx, Ly, T, R = 14, 10, 6, 200
    base = dict(lattice=3, Lx=Lx, Ly=Ly, n0=9.0, amp=30.0, mode_mx=1, init_weighted=1, omega_eff=1.7, seed=31)
    oj, om = B.lb_rates(base["omega_eff"])
    with B.LB(3, Lx, Ly, n0=9.0, amp=30.0, mode_mx=1, init_weighted=1, omega_j=oj, omega=om) as lb:
        lb.init()
        f0, _ = lb.get_state()
        lb.step(T)
        f, _ = lb.get_state()
    ora = OL.LB(3, Lx, Ly, omega_j=oj, omega=om)
    assert np.array_equal(f0, ora.init_mean(n0=9.0, amp=30.0, mode_mx=1, init_weighted=1))
    assert np.abs(f - ora.run(f0, T)).max() <= 8e-15 * (T + 10) * np.abs(f0).max()
    acc = np.zeros(f.shape)
    for r in range(R):
        with B.Lattice(**dict(base, replica=r)) as lat:
            lat.init()
            lat.step(T)
            acc += lat.get_state()[0]
    mean = acc / R
    chi2 = float((((mean - f) ** 2) / (f / R)).sum())
    assert stats.chi2.ppf(1e-6, f.size) < chi2 < stats.chi2.ppf(1 - 1e-6, f.size), chi2


@pytest.mark.parametrize("Lx,Ly,steps", [(3, 3, 9), (65536, 3, 3), (3, 2051, 4), (5, 7, 12)])
def test_extreme_extents(B, Lx, Ly, steps):
    """Smallest lattice (every diagonal wraps onto itself), very long rows, very tall
    columns: bit-exact against the oracle."""
    cfg = dict(lattice=3, Lx=Lx, Ly=Ly, n0=6.0, omega_eff=1.5, seed=Lx + Ly)
    ref = O.Lattice(**cfg)
    with B.Lattice(**cfg) as lat:
        lat.init()
        lat.step(steps)
        got, _ = lat.get_state()
    assert np.array_equal(got, ref.run(ref.init(), 0, steps))
