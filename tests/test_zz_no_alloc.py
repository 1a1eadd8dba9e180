"""ilg_observables_noalloc, the entry point for callers that cannot allocate
device memory when they need the observables (applications whose device memory
belongs to their own pool, real-time loops that must not wait on the allocator):
it must give the same mass,
projections, amplitudes and structure factors as ilg_observables on the same
state, call after call, although its scratch is one static device array shared
by every call.  This file is collected last so that a failure here never hides
the other tests."""
import ctypes

import numpy as np
import pytest

from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


def _device_copy(torch, B, lat):
    """The context's current state, copied into a device tensor the test owns."""
    buf = torch.empty(lat.size, dtype=torch.int16, device="cuda")
    lat.get_state_device(buf.data_ptr(), lat.size)
    torch.cuda.synchronize()
    return buf


MODES_2D = [(1, 0), (2, 0), (-3, 0), (0, 1), (0, 4)]


@pytest.mark.parametrize("lattice,Lx,Ly,modes", [
    (2, 96, 40, MODES_2D), (1, 256, 1, [(1, 0), (2, 0), (-3, 0)]), (2, 37, 53, MODES_2D),
    (3, 48, 20, MODES_2D),                                   # D2Q9: nine planes
    (2, 40, 24, []),                                         # mass only (no projection)
    (2, 32768, 3, [(m, 0) for m in range(1, 257)]),          # the side and mode limits
    (2, 3, 32768, [(0, 1), (0, 16384), (0, 32767)]),
])
def test_noalloc_matches_observables_twice(B, lattice, Lx, Ly, modes):
    torch = pytest.importorskip("torch")
    Q = {1: 3, 2: 5, 3: 9}[lattice]
    cfg = dict(lattice=lattice, Lx=Lx, Ly=Ly, omega_eff=1.7, seed=11)
    with B.Lattice(**cfg) as lat:
        for call, seed in enumerate((21, 22)):
            lat.set_state(inputs.random_state(Q, Ly, Lx, 30.0 + 10 * call, seed=seed), 0)
            lat.step(3)
            ref = lat.observables(modes)
            dev = _device_copy(torch, B, lat)
            got = B.observables_noalloc(lattice, Lx, Ly, dev.data_ptr(), modes)
            assert got["mass"] == ref["mass"], call
            for key in ("re", "im", "amp", "Sk"):
                scale = np.maximum(np.abs(ref[key]), 1.0)
                assert np.all(np.abs(got[key] - ref[key]) <= 1e-12 * scale), (call, key)


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    with pytest.raises(B.IlgError) as e:
        B.observables_noalloc(2, 65536, 8, 1, [(1, 0)])
    assert e.value.status == B.ILG_E_INVALID
    with pytest.raises(B.IlgError) as e:
        B.observables_noalloc(2, 64, 64, 1, [(1, 0)] * 257)
    assert e.value.status == B.ILG_E_INVALID
