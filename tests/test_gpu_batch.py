"""Batched D1Q3 rings (ilg_batch_*) against the oracle and against one context
per ring: every ring bit-identical, whatever the batch it runs in."""
import numpy as np
import pytest

import oracle as O
from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


def mixed_replicas(seed=4):
    """Rings of many lengths (one block-width and beyond, odd lengths), low and high
    occupations (fast and general collision paths), flip on and off, omega* = 1
    (every particle redistributed) and 0 (pure flip)."""
    Ls = [3, 17, 64, 255, 512, 513, 700, 1031, 2048, 4100]
    n0s = [4.0, 10.0, 30.0, 70.0, 120.0, 200.0]
    oms = [0.2, 0.7, 1.0, 1.3, 1.95, 2.0, 1.5]
    reps = []
    for i in range(len(Ls) * 2):
        reps.append(dict(lattice=1, Lx=Ls[i % len(Ls)], n0=n0s[i % len(n0s)], amp=0.0, mode_mx=0,
                         init_weighted=i % 2, omega_eff=oms[i % len(oms)], theta=0.3 + 0.05 * (i % 3),
                         seed=seed, replica=100 + i))
    return reps


def test_batch_init_and_run_match_oracle(B):
    reps = mixed_replicas()
    T = 40
    with B.Batch(reps) as bat:
        bat.init()
        for i, r in enumerate(reps):
            s, t = bat.get_state(i)
            assert t == 0 and np.array_equal(s, O.Lattice(**r).init()), i
        bat.run(T)
        for i, r in enumerate(reps):
            got, t = bat.get_state(i)
            ref = O.Lattice(**r)
            assert t == T
            assert np.array_equal(got, ref.run(ref.init(), 0, T)), (i, r)


def test_batch_longest_rings_match_oracle(B):
    """Rings at the length limit (10240 nodes, the ring and its copy in shared memory
    beside the packed tables and 1024 threads' extension words) next to a short one,
    through every block shape the autotuner times."""
    reps = [dict(lattice=1, Lx=L, n0=n0, amp=8.0, mode_mx=1, omega_eff=w, seed=11, replica=i)
            for i, (L, n0, w) in enumerate([(10240, 20.0, 1.5), (10233, 60.0, 0.8), (100, 10.0, 1.9)])]
    with B.Batch(reps) as bat:
        bat.init()
        bat.run(6)
        tun = bat.autotune(3)
        assert all(v is not None for v in tun["ms_per_step"].values())
        bat.run(4)
        for i, r in enumerate(reps):
            got, t = bat.get_state(i)
            ref = O.Lattice(**r)
            assert t == 10 and np.array_equal(got, ref.run(ref.init(), 0, 10)), i
    with pytest.raises(B.IlgError):
        B.Batch([dict(lattice=1, Lx=10241, seed=1)])


def test_batch_mixed_samplers_match_oracle(B):
    """Rings with the particle sampler next to rings with the binomial sampler."""
    reps = [dict(lattice=1, Lx=L, n0=n0, amp=0.0, omega_eff=w, seed=8, replica=i, sampler=i % 2)
            for i, (L, n0, w) in enumerate([(40, 10.0, 1.5), (40, 10.0, 1.5), (130, 60.0, 0.7), (257, 25.0, 1.9),
                                            (600, 5.0, 1.0), (64, 100.0, 1.2)])]
    with B.Batch(reps) as bat:
        bat.init()
        bat.run(15)
        for i, r in enumerate(reps):
            got, t = bat.get_state(i)
            ref = O.Lattice(**r)
            assert t == 15 and np.array_equal(got, ref.run(ref.init(), 0, 15)), i


def test_batch_equals_single_contexts(B):
    reps = mixed_replicas(seed=9)[:8]
    states = [inputs.random_state(3, 1, r["Lx"], r["n0"], seed=50 + i) for i, r in enumerate(reps)]
    with B.Batch(reps) as bat:
        for i, s in enumerate(states):
            bat.set_state(i, s, 7)
        bat.run(25)
        bat.run(25)
        got = [bat.get_state(i) for i in range(len(reps))]
    for i, r in enumerate(reps):
        with B.Lattice(**r) as lat:
            lat.set_state(states[i], 7)
            lat.step(50)
            ref, t = lat.get_state()
        assert got[i][1] == t == 57 and np.array_equal(got[i][0], ref), i


def test_batch_record_and_observables(B):
    """Amplitude of mode 1 after every step (the Fig. 1 observable, Sec. V)."""
    reps = [dict(lattice=1, Lx=L, n0=100.0 / 3.0, amp=100.0, mode_mx=1, init_weighted=1,
                 omega_eff=w, seed=3, replica=i) for i, (L, w) in enumerate([(320, 1.5), (256, 0.8), (101, 1.9)])]
    T = 30
    with B.Batch(reps) as bat:
        bat.init()
        rec = bat.run(T, record_mode=1)
        mass, amp = bat.observables(1)
    for i, r in enumerate(reps):
        ref = O.Lattice(**r)
        s = ref.init()
        for t in range(T):
            s = ref.step(s, t)
            M, _, _, res = ref.observables(s, [(1, 0)])
            tol = 1e-12 * res[0]["scale"] / (r["Lx"] / 2)
            assert abs(rec[i, t] - res[0]["amp"]) <= tol, (i, t)
        assert mass[i] == M
        assert abs(amp[i] - res[0]["amp"]) <= tol


def test_batch_overflow_stops_only_that_ring(B):
    reps = [dict(lattice=1, Lx=40, omega_eff=1.0, seed=2, replica=i) for i in range(3)]
    states = [inputs.random_state(3, 1, 40, 5.0, seed=i) for i in range(3)]
    states[1][:, 0, 10] = 40000         # omega* = 1 sends about 2/3 of 120000 to rest
    ref = O.Lattice(**reps[1])
    cur, fail_t = states[1].copy(), None
    for t in range(5):
        try:
            cur = ref.step(cur, t)
        except OverflowError:
            fail_t = t
            break
    assert fail_t is not None
    with B.Batch(reps) as bat:
        for i, s in enumerate(states):
            bat.set_state(i, s, 0)
        with pytest.raises(B.IlgError) as e:
            bat.run(5)
        assert e.value.status == B.ILG_E_OVERFLOW
        got1, t1 = bat.get_state(1)
        got0, t0 = bat.get_state(0)
    assert t1 == fail_t and np.array_equal(got1, cur)
    r0 = O.Lattice(**reps[0])
    assert t0 == 5 and np.array_equal(got0, r0.run(states[0], 0, 5))


def test_batch_workload_full_size(B):
    """The 4096-ring workload (lengths log-uniform in [64, 8192], occupations
    uniform in [5, 200], omega_eff uniform in [0.2, 1.95], seed 4) for 5000 steps in
    the launch the benchmark times: mass of every ring conserved exactly, and the
    three shortest rings and a window of the longest equal to the oracle."""
    reps = inputs.batch_replicas()
    T = 5000
    with B.Batch(reps) as bat:
        bat.init()
        m0, _ = bat.observables(1)
        bat.run(T)
        m1, _ = bat.observables(1)
        assert np.array_equal(m0, m1)
        Ls = np.array([r["Lx"] for r in reps])
        for i in list(np.argsort(Ls, kind="stable")[:3]):
            got, t = bat.get_state(int(i))
            ref = O.Lattice(**reps[i])
            assert t == T and np.array_equal(got, ref.run(ref.init(), 0, T)), i
        big = int(np.argmax(Ls))
        got, _ = bat.get_state(big)
    ref = O.Lattice(**reps[big])
    L = reps[big]["Lx"]
    x0, w = L - 3, 6
    win = ref.window(x0, 0, w, 1, T)      # light cone wider than the ring: wraps around it
    xs = [(x0 + k) % L for k in range(w)]
    assert np.array_equal(got[:, :, xs], win)


def test_run_record_states_and_amplitudes_every_step(B):
    """ilg_batch_run_record: the state of every ring after every step equals the
    oracle's step by step, and the amplitude record equals ilg_batch_run's; rings of
    three lengths (the ring workload's L = 256, an odd length, one above a block)."""
    reps = [dict(inputs.RING_D1Q3, replica=0),
            dict(lattice=1, Lx=37, n0=12.0, amp=3.0, mode_mx=1, omega_eff=0.7, seed=1, replica=1),
            dict(lattice=1, Lx=1100, n0=8.0, amp=2.0, mode_mx=2, omega_eff=1.9, seed=1, replica=2)]
    reps = [{k: v for k, v in r.items() if k != "steps"} for r in reps]
    T = 25
    with B.Batch(reps) as bat:
        bat.init()
        amp, states = bat.run_record(T, record_mode=1)
        got_end = [bat.get_state(i)[0] for i in range(len(reps))]
    with B.Batch(reps) as bat:
        bat.init()
        amp_plain = bat.run(T, record_mode=1)
    assert np.array_equal(amp, amp_plain)
    for i, r in enumerate(reps):
        ref = O.Lattice(**r)
        s = ref.init()
        for step in range(T):
            s = ref.step(s, step)
            assert np.array_equal(states[i][step], s), (i, step)
        assert np.array_equal(states[i][T - 1], got_end[i])
