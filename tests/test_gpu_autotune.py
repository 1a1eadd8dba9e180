"""Autotuner (ilg_autotune, ilg_batch_autotune) and the launch shapes it chooses
between: every shape gives the oracle's bits, tuning leaves the state and the step
counter alone, and candidates that cannot apply are reported as such."""
import numpy as np
import pytest

import oracle as O
from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


@pytest.mark.parametrize("omega", [1.7, 0.6])
@pytest.mark.parametrize("kernel", [0, 1, 2, 5, 6, 7, -1])
@pytest.mark.parametrize("lattice,Lx,Ly,mean,hot", [(2, 96, 40, 10.0, 3), (2, 100, 23, 8.0, 0), (1, 2052, 1, 20.0, 2),
                                                    (2, 2056, 9, 6.0, 0), (2, 8200, 3, 6.0, 1),
                                                    (1, 16392, 1, 20.0, 2)])
def test_every_shape_is_bit_exact(B, kernel, lattice, Lx, Ly, mean, hot, omega):
    """8- and 4-node vectors in row tiles, 8-node vectors in warp segments (rows of 96,
    100, 2052, 2056 nodes: several tiles, ragged tails, occupations that need the
    general pass; rows of 8200 and 16392 nodes: segments of 8192 nodes and a one-vector
    remainder), 4-node vectors in warp segments (the row split into segments whose
    end values are stored by the warp that owns them), node-parallel, default; with
    the flip (omega_eff 1.7) and without it (0.6: the kernels' other compile-time
    plane order)."""
    Q = 3 if lattice == 1 else 5
    s0 = inputs.random_state(Q, Ly, Lx, mean, seed=Lx + Ly, hot=hot, hot_value=500)
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, omega_eff=omega, seed=9, replica=1)
    with B.Lattice(**cfg) as lat:
        lat.set_step_kernel(kernel)
        lat.set_state(s0, 3)
        lat.step(9)
        got, t = lat.get_state()
    assert t == 12 and np.array_equal(got, O.Lattice(**cfg).run(s0, 3, 9))


def test_autotune_keeps_state_and_results(B):
    cfg = dict(lattice=2, Lx=256, Ly=96, n0=10.0, amp=4.0, mode_mx=1, omega_eff=1.8, seed=4)
    ref = O.Lattice(**cfg)
    with B.Lattice(**cfg) as lat:
        lat.init()
        lat.step(3)
        before, t0 = lat.get_state()
        tun = lat.autotune(6)
        after, t1 = lat.get_state()
        assert t0 == t1 == 3 and np.array_equal(before, after)
        assert set(tun["ms_per_step"]) == {"vec8", "vec4", "node", "tb2", "tb4", "seg8", "warpv8", "warpv4"}
        assert all(v is not None and v > 0 for v in tun["ms_per_step"].values())
        assert tun["ms_per_step"][tun["choice"]] == min(tun["ms_per_step"].values())
        lat.step(9)
        got, t = lat.get_state()
    assert t == 12 and np.array_equal(got, ref.run(ref.init(), 0, 12))


@pytest.mark.parametrize("cfg,applicable", [
    (dict(lattice=1, Lx=1028, n0=10.0), {"vec8": False, "vec4": True, "node": True, "tb2": False, "tb4": False,
                                         "seg8": False, "warpv8": False, "warpv4": True}),
    (dict(lattice=3, Lx=64, Ly=32, n0=6.0), {"vec8": False, "vec4": False, "node": True, "tb2": False, "tb4": False,
                                              "seg8": False, "warpv8": True, "warpv4": True}),
    (dict(lattice=3, Lx=66, Ly=8, n0=6.0), {"vec8": False, "vec4": False, "node": True, "tb2": False, "tb4": False,
                                             "seg8": False, "warpv8": False, "warpv4": False}),
    (dict(lattice=3, Lx=64, Ly=8, n0=6.0, sampler=1), {"vec8": False, "vec4": False, "node": True, "tb2": False,
                                                        "tb4": False, "seg8": False, "warpv8": False,
                                                        "warpv4": False}),
    (dict(lattice=2, Lx=64, Ly=32, n0=80.0), {"vec8": False, "vec4": False, "node": True, "tb2": True, "tb4": True,
                                              "seg8": False, "warpv8": False, "warpv4": False}),
    (dict(lattice=2, Lx=1024, Ly=24, n0=10.0), {"vec8": True, "vec4": True, "node": True, "tb2": True, "tb4": True,
                                               "seg8": True, "warpv8": True, "warpv4": True}),
    (dict(lattice=2, Lx=1020, Ly=6, n0=10.0), {"vec8": False, "vec4": True, "node": True, "tb2": True, "tb4": True,
                                              "seg8": False, "warpv8": False, "warpv4": True}),
])
def test_autotune_candidates(B, cfg, applicable):
    with B.Lattice(omega_eff=1.5, seed=2, **cfg) as lat:
        lat.init()
        tun = lat.autotune(4)
        for name, ok in applicable.items():
            assert (tun["ms_per_step"][name] is not None) == ok, name
        lat.step(3)
        got, _ = lat.get_state()
    ref = O.Lattice(omega_eff=1.5, seed=2, **cfg)
    assert np.array_equal(got, ref.run(ref.init(), 0, 3))


def test_batch_autotune(B):
    reps = [dict(lattice=1, Lx=L, n0=n0, omega_eff=w, seed=6, replica=i)
            for i, (L, n0, w) in enumerate([(40, 10.0, 1.5), (300, 60.0, 0.8), (1500, 20.0, 1.9), (64, 150.0, 1.2),
                                            (2100, 5.0, 1.0)])]
    with B.Batch(reps) as bat:
        bat.init()
        bat.run(4)
        before = [bat.get_state(i) for i in range(len(reps))]
        tun = bat.autotune(10)
        after = [bat.get_state(i) for i in range(len(reps))]
        for (a, ta), (b, tb) in zip(before, after):
            assert ta == tb == 4 and np.array_equal(a, b)
        assert tun["threads"] in (256, 512, 1024)
        bat.run(11)
        for i, r in enumerate(reps):
            got, t = bat.get_state(i)
            ref = O.Lattice(**r)
            assert t == 15 and np.array_equal(got, ref.run(ref.init(), 0, 15)), i
