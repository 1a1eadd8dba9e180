"""Temporal blocking (several steps per launch in shared-memory tiles with a
recomputed halo) gives the same bits as single steps and as the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


@pytest.mark.parametrize("Lx,Ly,depth,steps", [(96, 96, 2, 8), (100, 70, 3, 11), (37, 29, 4, 9),
                                               (200, 50, 8, 17), (48, 48, 2, 5), (20, 130, 5, 10)])
def test_tb_equals_single_steps_and_oracle(B, Lx, Ly, depth, steps):
    s0 = inputs.random_state(5, Ly, Lx, 14.0, seed=Lx + Ly, hot=6, hot_value=300)
    cfg = dict(lattice=2, Lx=Lx, Ly=Ly, omega_eff=1.7, seed=12, replica=3)
    with B.Lattice(**cfg) as lat:
        lat.set_temporal_blocking(depth)
        lat.set_state(s0, 40)
        lat.step(steps)
        got, t = lat.get_state()
    assert t == 40 + steps
    assert np.array_equal(got, O.Lattice(**cfg).run(s0, 40, steps))


def test_tb_high_occupation(B):
    """Mean occupation 60 per velocity: every node takes the general collision,
    with more extension words than the per-thread buffer holds."""
    Lx, Ly = 70, 52
    cfg = dict(lattice=2, Lx=Lx, Ly=Ly, n0=60.0, amp=25.0, mode_mx=1, omega_eff=1.0, seed=21, replica=5)
    ref = O.Lattice(**cfg)
    s0 = ref.init()
    with B.Lattice(**cfg) as lat:
        lat.set_temporal_blocking(3)
        lat.init()
        lat.step(7)
        got, t = lat.get_state()
    assert t == 7 and np.array_equal(got, ref.run(s0, 0, 7))


def test_tb_full_size_window(B):
    """16384^2 workload, 40 steps at depth 4 against single steps (whole state)."""
    cfg = {k: v for k, v in inputs.LARGE_D2Q5.items() if k != "steps"}
    with B.Lattice(**cfg) as a, B.Lattice(**cfg) as b:
        a.init()
        b.init()
        a.set_temporal_blocking(4)
        a.step(40)
        b.step(40)
        sa = np.empty(a.shape, np.uint16)
        sb = np.empty(b.shape, np.uint16)
        a.get_state(sa)
        b.get_state(sb)
    assert np.array_equal(sa, sb)


def test_tb_overflow_keeps_launch_input(B):
    Lx = Ly = 20
    s = inputs.random_state(5, Ly, Lx, 3.0, seed=8)
    s[:, 5, 7] = 40000
    cfg = dict(lattice=2, Lx=Lx, Ly=Ly, omega_eff=1.0, seed=4)
    ref = O.Lattice(**cfg)
    cur, fail_t = s.copy(), None
    for t in range(12):
        try:
            cur = ref.step(cur, t)
        except OverflowError:
            fail_t = t
            break
    assert fail_t is not None
    depth = 3
    launch_t = (fail_t // depth) * depth           # the failing launch starts here
    expect = ref.run(s, 0, launch_t)
    with B.Lattice(**cfg) as lat:
        lat.set_temporal_blocking(depth)
        lat.set_state(s, 0)
        with pytest.raises(B.IlgError) as e:
            lat.step(12)
        assert e.value.status == B.ILG_E_OVERFLOW
        got, t = lat.get_state()
    assert t == launch_t and np.array_equal(got, expect)


def test_tb_rejected_on_d1q3(B):
    with B.Lattice(lattice=1, Lx=64) as lat:
        with pytest.raises(B.IlgError):
            lat.set_temporal_blocking(2)
