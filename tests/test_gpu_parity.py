"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Integer results (states, sums, Philox words, tables) must match bit for bit;
the double-precision projections to 1e-12 relative to sum_x |D(x)| / L (their
condition scale: device sincospi and host sin/cos differ by an ulp or so, and
the device sum is compensated).  Inputs are seeded and synthetic.
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


def gpu_run(B, cfg, steps, state=None, t0=0):
    with B.Lattice(**cfg) as lat:
        if state is None:
            lat.init()
        else:
            lat.set_state(state, t0)
        lat.step(steps)
        out, t = lat.get_state()
    assert t == t0 + steps
    return out


# ---------------------------------------------------------------- building blocks

def test_philox_device_matches_oracle(B):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 2, 3, 4], [0xFFFFFFFF] * 4, [7, 0, 0, 0x03000001]]
    for seed in (0, 3, 0xFEDCBA9876543210):
        out = B.philox(ctr, seed)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i in list(range(64)) + list(rng.integers(0, len(ctr), 200)):
            assert np.array_equal(out[i], O.philox(ctr[i], key)), (seed, i)


@pytest.mark.parametrize("p", [1e-9, 0.1, 0.2, 1.0 / 3.0, 0.5, 0.9, 0.999999])
def test_binomial_tables_match(B, p):
    P = O.quantise(p)
    assert np.array_equal(B.binomial_table(P), O.binomial_table(P))
    thr, al = B.alias_table(P)
    othr, oal = O.alias_table(P)
    assert np.array_equal(thr, othr) and np.array_equal(al, oal.astype(np.uint32))


@pytest.mark.parametrize("lam", [0.0, 1e-3, 0.5, 10.0, 30.0, 50.0 + 4.0 * 0.7071067811865476, 200.0, 699.0])
def test_poisson_tables_match(B, lam):
    assert np.array_equal(B.poisson_table(lam), O.poisson_table(lam))


# ---------------------------------------------------------------- initial state

INIT_CASES = [
    dict(lattice=1, Lx=256, n0=30.0, amp=10.0, mode_mx=1, init_weighted=0, seed=1),
    dict(lattice=1, Lx=320, n0=100.0 / 3.0, amp=100.0, mode_mx=1, init_weighted=1, seed=5, replica=77),
    dict(lattice=2, Lx=96, Ly=64, n0=50.0, amp=20.0, mode_mx=1, init_weighted=0, seed=2),
    dict(lattice=2, Lx=37, Ly=29, n0=7.5, amp=6.0, mode_my=-3, init_weighted=1, seed=9, theta=0.4),
    dict(lattice=2, Lx=130, Ly=33, n0=10.0, seed=3, replica=2),
]


@pytest.mark.parametrize("cfg", INIT_CASES)
def test_init_bit_exact(B, cfg):
    with B.Lattice(**cfg) as lat:
        lat.init()
        got, t = lat.get_state()
    assert t == 0
    assert np.array_equal(got, O.Lattice(**cfg).init())


# ---------------------------------------------------------------- time step

STEP_CASES = [
    # lattice, Lx, Ly, omega_eff, theta, mean, hot
    (1, 257, 1, 1.5, 1.0 / 3.0, 30.0, 0),
    (1, 1000, 1, 0.5, 1.0 / 3.0, 90.0, 10),
    (1, 64, 1, 1.95, 0.6, 200.0, 0),
    (1, 9, 1, 2.0, 1.0 / 3.0, 5.0, 0),
    (2, 37, 29, 1.8, 1.0 / 3.0, 10.0, 0),
    (2, 64, 48, 1.0, 1.0 / 3.0, 50.0, 0),
    (2, 130, 70, 0.5, 1.0 / 3.0, 20.0, 25),
    (2, 33, 17, 1.9, 0.5, 12.0, 0),
    (2, 16, 16, 1e-12, 1.0 / 3.0, 8.0, 0),
    (2, 24, 40, 1.3, 0.45, 60.0, 40),
    # row-tiled kernel: rows of 1, 2 and 3 tiles with ragged last tiles, one-vector rows
    (2, 2344, 5, 1.8, 1.0 / 3.0, 10.0, 30),
    (1, 4104, 1, 1.4, 1.0 / 3.0, 70.0, 12),
    (2, 8, 6, 1.6, 1.0 / 3.0, 20.0, 0),
    (1, 8, 1, 0.9, 1.0 / 3.0, 40.0, 0),
    (2, 2048, 3, 0.7, 1.0 / 3.0, 30.0, 0),
]


@pytest.mark.parametrize("lattice,Lx,Ly,omega,theta,mean,hot", STEP_CASES)
def test_step_bit_exact(B, lattice, Lx, Ly, omega, theta, mean, hot):
    Q = 3 if lattice == 1 else 5
    s0 = inputs.random_state(Q, Ly, Lx, mean, seed=Lx * 7 + Ly, hot=hot, hot_value=900)
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, omega_eff=omega, theta=theta, seed=Lx + 1000 * Ly, replica=5)
    t0, steps = 17, 12
    got = gpu_run(B, cfg, steps, state=s0, t0=t0)
    ref = O.Lattice(**cfg).run(s0, t0, steps)
    assert np.array_equal(got, ref)


def test_ring_d1q3_full_workload_bit_exact(B):
    """D1Q3 ring L=256, mean 30 + sine amplitude 10, omega_eff 1.5, 2000 steps, seed 1:
    the full workload, every step's amplitude and the final state."""
    cfg = {k: v for k, v in inputs.RING_D1Q3.items() if k != "steps"}
    ref = O.Lattice(**cfg)
    s = ref.init()
    with B.Lattice(**cfg) as lat:
        lat.init()
        for block in range(20):
            lat.step(100)
            s = ref.run(s, block * 100, 100)
            got, t = lat.get_state()
            assert np.array_equal(got, s), t
            obs = lat.observables([(1, 0)], col_sums=True)
            M, col, _, res = ref.observables(s, [(1, 0)])
            assert obs["mass"] == M and np.array_equal(obs["col"], col)
            assert abs(obs["amp"][0] - res[0]["amp"]) <= 1e-12 * res[0]["scale"] / (cfg["Lx"] / 2)


def test_sweep_d2q5_reduced_bit_exact(B):
    for c in inputs.SWEEP_D2Q5:
        cfg = inputs.scaled({k: v for k, v in c.items() if k != "steps"}, Lx=128, Ly=96)
        ref = O.Lattice(**cfg)
        with B.Lattice(**cfg) as lat:
            lat.init()
            lat.step(40)
            got, _ = lat.get_state()
        assert np.array_equal(got, ref.run(ref.init(), 0, 40)), c["omega_eff"]


# ---------------------------------------------------------------- observables

@pytest.mark.parametrize("lattice,Lx,Ly", [(1, 256, 1), (2, 96, 40), (2, 37, 53)])
def test_observables(B, lattice, Lx, Ly):
    Q = 3 if lattice == 1 else 5
    s = inputs.random_state(Q, Ly, Lx, 25.0, seed=5, hot=3, hot_value=60000)
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, omega_eff=1.2, seed=1)
    modes = [(1, 0), (2, 0), (-3, 0), (Lx // 2 - 1, 0)] + ([(0, 1), (0, 5)] if lattice == 2 else [])
    with B.Lattice(**cfg) as lat:
        lat.set_state(s, 4)
        obs = lat.observables(modes, col_sums=True, row_sums=True)
    M, col, row, res = O.Lattice(**cfg).observables(s, modes)
    assert obs["t"] == 4 and obs["mass"] == M
    assert np.array_equal(obs["col"], col) and np.array_equal(obs["row"], row)
    K = Lx * Ly
    for i, r in enumerate(res):
        tol = 1e-12 * r["scale"]
        assert abs(obs["re"][i] - r["re"]) <= tol
        assert abs(obs["im"][i] - r["im"]) <= tol
        assert abs(obs["amp"][i] - r["amp"]) <= tol / (K / 2)
        assert abs(obs["Sk"][i] - r["Sk"]) <= 2 * tol * (abs(r["re"]) + abs(r["im"]) + tol) / K


# ---------------------------------------------------------------- errors and rollback

def test_overflow_rolls_back(B):
    """omega* = 1 puts about w_0 N of every node into the rest velocity; a node
    holding 5 x 40000 particles overflows uint16 there.  The oracle names the
    failing step; the context must hold the state at that step."""
    Lx, Ly = 20, 12
    s = inputs.random_state(5, Ly, Lx, 3.0, seed=8)
    s[:, 5, 7] = 40000
    cfg = dict(lattice=2, Lx=Lx, Ly=Ly, omega_eff=1.0, seed=4)
    ref = O.Lattice(**cfg)
    cur, fail_t = s.copy(), None
    for t in range(10):
        try:
            cur = ref.step(cur, t)
        except OverflowError:
            fail_t = t
            break
    assert fail_t is not None
    with B.Lattice(**cfg) as lat:
        lat.set_state(s, 0)
        with pytest.raises(B.IlgError) as e:
            lat.step(10)
        assert e.value.status == B.ILG_E_OVERFLOW
        got, t = lat.get_state()
    assert t == fail_t
    assert np.array_equal(got, cur)


@pytest.mark.parametrize("kernel", [6, 7])
@pytest.mark.parametrize("lattice,Lx,Ly", [(1, 4096, 1), (2, 256, 64), (3, 256, 32)])
def test_overflow_in_staged_warp_step(B, kernel, lattice, Lx, Ly):
    """A node holding 65535 particles in every velocity overflows through the staged
    warp step (its general collision: the fast one refuses the node) on a lattice whose
    mean stays low enough for that kernel; the context reports the overflow and holds
    the state of the step that failed, as the oracle names it."""
    Q = {1: 3, 2: 5, 3: 9}[lattice]
    s = inputs.random_state(Q, Ly, Lx, 3.0, seed=Lx + Q)
    s[:, Ly // 2, 37] = 65535
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, omega_eff=1.9, seed=5)
    ref = O.Lattice(**cfg)
    cur, fail_t = s.copy(), None
    for t in range(6):
        try:
            cur = ref.step(cur, t)
        except OverflowError:
            fail_t = t
            break
    assert fail_t is not None
    with B.Lattice(**cfg) as lat:
        lat.set_step_kernel(kernel)
        lat.set_state(s, 0)
        with pytest.raises(B.IlgError) as e:
            lat.step(6)
        assert e.value.status == B.ILG_E_OVERFLOW
        got, t = lat.get_state()
    assert t == fail_t and np.array_equal(got, cur)


def test_invalid_arguments(B):
    bad = [dict(lattice=3, Lx=10), dict(lattice=1, Lx=2), dict(lattice=2, Lx=10, Ly=2),
           dict(lattice=1, Lx=10, omega_eff=0.0), dict(lattice=1, Lx=10, omega_eff=2.5),
           dict(lattice=2, Lx=10, Ly=10, theta=0.6), dict(lattice=1, Lx=10, n0=-1.0),
           dict(lattice=2, Lx=10, Ly=10, mode_mx=1, mode_my=1)]
    for cfg in bad:
        with pytest.raises(B.IlgError) as e:
            B.Lattice(**cfg)
        assert e.value.status == B.ILG_E_INVALID, cfg
    with B.Lattice(lattice=1, Lx=10) as lat:
        with pytest.raises(B.IlgError) as e:
            lat.step(1)
        assert e.value.status == B.ILG_E_STATE
        with pytest.raises(ValueError):
            lat.set_state(np.zeros(7, np.uint16))
    with B.Lattice(lattice=1, Lx=64, n0=1.0, amp=10.0, mode_mx=1) as lat:
        with pytest.raises(B.IlgError) as e:
            lat.init()
        assert e.value.status == B.ILG_E_INVALID


def test_checkpoint_resume(B):
    cfg = dict(lattice=2, Lx=48, Ly=40, n0=9.0, omega_eff=1.7, seed=77)
    with B.Lattice(**cfg) as a:
        a.init()
        a.step(30)
        full, t = a.get_state()
    with B.Lattice(**cfg) as b:
        b.init()
        b.step(13)
        mid, tm = b.get_state()
    with B.Lattice(**cfg) as c:
        c.set_state(mid, tm)
        c.step(17)
        res, tr = c.get_state()
    assert t == tr == 30 and np.array_equal(full, res)


# ---------------------------------------------------------------- full-size light cones

def test_large_d2q5_light_cone_full_size(B):
    """16384^2, mean 10 per velocity, omega_eff 1.8, 500 steps (the throughput
    workload, same kernels and launch shape): 12 x 12 windows at t = 500 from the
    oracle's own initial state of their light cones, one across the periodic seam of
    the rows and one across the middle of the rows (where the default kernel's two
    8192-node segments of a row meet); plus exact mass."""
    cfg = {k: v for k, v in inputs.LARGE_D2Q5.items() if k != "steps"}
    steps = inputs.LARGE_D2Q5["steps"]
    x0, y0, w = 16384 - 5, 9000, 12
    with B.Lattice(**cfg) as lat:
        lat.init()
        m0 = lat.observables()["mass"]
        lat.step(steps)
        obs = lat.observables([(1, 0), (2, 0)])
        state = np.empty(lat.shape, np.uint16)
        lat.get_state(state)
    assert obs["mass"] == m0 and obs["t"] == steps
    ref = O.Lattice(**cfg)
    for x0, y0 in ((x0, y0), (8192 - 6, 3000)):
        win = ref.window(x0, y0, w, w, steps)
        xs = [(x0 + i) % 16384 for i in range(w)]
        assert np.array_equal(state[:, y0:y0 + w][:, :, xs], win), (x0, y0)


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("lattice,Lx,Ly,steps", [(2, 3, 3, 7), (2, 16, 3, 9), (2, 65536, 3, 3), (2, 8, 2051, 4),
                                                 (1, 3, 1, 15), (1, 65544, 1, 5)])
def test_extreme_shapes(B, lattice, Lx, Ly, steps):
    Q = 3 if lattice == 1 else 5
    s0 = inputs.random_state(Q, Ly, Lx, 20.0, seed=Lx % 1000 + Ly)
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, omega_eff=1.55, seed=0xFFFFFFFF00000001, replica=0xFFFFFFFF)
    got = gpu_run(B, cfg, steps, state=s0, t0=3)
    assert np.array_equal(got, O.Lattice(**cfg).run(s0, 3, steps))


def test_occupations_near_the_limit(B):
    """Nodes holding up to 65535 particles in total never overflow (mass is
    conserved per node); pure flip moves them untouched."""
    Lx, Ly = 40, 24
    s = np.zeros((5, Ly, Lx), np.uint16)
    s[0, 3, 5] = 65535
    s[1, 10, 10] = 30000
    s[2, 10, 10] = 35535
    s[:, 20, 30] = [13107] * 5
    for omega in (0.5, 1.0, 1.5, 2.0):
        cfg = dict(lattice=2, Lx=Lx, Ly=Ly, omega_eff=omega, seed=77)
        got = gpu_run(B, cfg, 6, state=s, t0=0)
        assert np.array_equal(got, O.Lattice(**cfg).run(s, 0, 6)), omega


def test_step_counter_limit(B):
    s0 = inputs.random_state(3, 1, 32, 10.0, seed=1)
    cfg = dict(lattice=1, Lx=32, omega_eff=1.2, seed=2)
    t0 = (1 << 32) - 20
    got = gpu_run(B, cfg, 10, state=s0, t0=t0)
    assert np.array_equal(got, O.Lattice(**cfg).run(s0, t0, 10))
    with B.Lattice(**cfg) as lat:
        lat.set_state(s0, t0)
        with pytest.raises(B.IlgError) as e:
            lat.step(20)
        assert e.value.status == B.ILG_E_INVALID


def test_init_largest_mean(B):
    cfg = dict(lattice=2, Lx=64, Ly=16, n0=660.0, amp=150.0, mode_mx=2, init_weighted=0, seed=6)
    with B.Lattice(**cfg) as lat:
        lat.init()
        got, _ = lat.get_state()
    assert np.array_equal(got, O.Lattice(**cfg).init())


@pytest.mark.parametrize("lattice,Lx,Ly,n0,omega", [(2, 64, 16, 660.0, 1.0), (1, 512, 1, 660.0, 1.0),
                                                    (2, 40, 24, 120.0, 1.5), (1, 96, 1, 300.0, 0.6)])
def test_step_very_high_occupation(B, lattice, Lx, Ly, n0, omega):
    """Hundreds of particles per velocity: the general collision needs more
    extension words than a thread's shared-memory buffer holds and refills it."""
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, n0=n0, amp=n0 / 20, mode_mx=1, init_weighted=0,
               omega_eff=omega, seed=31, replica=4)
    ref = O.Lattice(**cfg)
    assert np.array_equal(gpu_run(B, cfg, 6), ref.run(ref.init(), 0, 6))


def test_set_state_high_mass_takes_general_path(B):
    """A state set from the host with a high mean (decided on the device) after an
    init with a low one: same bits as the oracle either way."""
    cfg = dict(lattice=2, Lx=64, Ly=32, n0=5.0, omega_eff=1.2, seed=8)
    s_hi = inputs.random_state(5, 32, 64, 90.0, seed=3)
    with B.Lattice(**cfg) as lat:
        lat.init()
        lat.step(3)
        lat.set_state(s_hi, 11)
        lat.step(5)
        got, t = lat.get_state()
    assert t == 16 and np.array_equal(got, O.Lattice(**cfg).run(s_hi, 11, 5))


@pytest.mark.parametrize("lattice,Lx,Ly,omega", [(1, 128, 1, 1.0), (2, 64, 24, 1.5), (2, 37, 29, 0.7),
                                                 (3, 24, 20, 1.0), (3, 19, 13, 1.6)])
def test_chunk_boundary_occupations(B, lattice, Lx, Ly, omega):
    """Occupations on both sides of the alias rows' limit (63 trials per draw) and of
    the 32-particle direction groups: the fast path's edges, one and two extension
    chunks, and their mix within a row and a vector."""
    Q = {1: 3, 2: 5, 3: 9}[lattice]
    edges = np.array([0, 1, 31, 32, 33, 62, 63, 64, 65, 125, 126, 127, 128, 189, 190], dtype=np.uint16)
    s0 = np.random.default_rng(lattice * 7 + Lx).choice(edges, size=(Q, Ly, Lx)).astype(np.uint16)
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, n0=10.0, omega_eff=omega, seed=12, replica=3)
    got = gpu_run(B, cfg, 3, state=s0, t0=5)
    assert np.array_equal(got, O.Lattice(**cfg).run(s0, 5, 3))


# ---------------------------------------------------------------- particle sampler
PARTICLE_CASES = [
    # lattice, Lx, Ly, omega_eff, mean, hot
    (1, 200, 1, 1.5, 20.0, 2),
    (1, 64, 1, 0.6, 5.0, 0),
    (2, 64, 24, 1.8, 10.0, 3),     # rows a multiple of 8: still the node-parallel kernel
    (2, 37, 29, 1.0, 12.0, 0),     # omega* = 1: no particle stays
    (2, 40, 16, 2.0, 9.0, 0),      # omega* = 0: every particle stays (pure flip)
    (2, 33, 21, 0.3, 60.0, 2),
]


@pytest.mark.parametrize("lattice,Lx,Ly,omega,mean,hot", PARTICLE_CASES)
def test_particle_sampler_bit_exact(B, lattice, Lx, Ly, omega, mean, hot):
    Q = 3 if lattice == 1 else 5
    s0 = inputs.random_state(Q, Ly, Lx, mean, seed=Lx + 3 * Ly, hot=hot, hot_value=700)
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, omega_eff=omega, seed=41, replica=3, sampler=1)
    got = gpu_run(B, cfg, 7, state=s0, t0=12)
    assert np.array_equal(got, O.Lattice(**cfg).run(s0, 12, 7))


def test_particle_sampler_init_and_temporal_blocking(B):
    cfg = dict(lattice=2, Lx=50, Ly=44, n0=8.0, amp=6.0, mode_mx=1, omega_eff=1.4, seed=5, sampler=1)
    ref = O.Lattice(**cfg)
    with B.Lattice(**cfg) as lat:
        lat.set_temporal_blocking(3)
        lat.init()
        lat.step(7)
        got, t = lat.get_state()
    assert t == 7 and np.array_equal(got, ref.run(ref.init(), 0, 7))


def test_sampler_value_checked(B):
    with pytest.raises(B.IlgError) as e:
        B.Lattice(lattice=2, Lx=16, Ly=16, sampler=2)
    assert e.value.status == B.ILG_E_INVALID
