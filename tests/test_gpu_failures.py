"""Error paths, made to fail on the host: ilg_inject_alloc_failure makes one of the
library's device allocations report failure (no allocator call, no GPU fault).
Every create call must return ILG_E_OOM with a message naming the failure, free
what it had allocated (device memory returns to where it was), and leave the
library working for the next call."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


@pytest.fixture()
def torch():
    t = pytest.importorskip("torch")
    t.cuda.init()
    return t


def free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


CFG = dict(lattice=2, Lx=512, Ly=256, n0=10.0, omega_eff=1.8, seed=5)


def test_every_allocation_of_a_context_can_fail(B, torch):
    """Each of ilg_create's device allocations in turn reports failure: ILG_E_OOM,
    ilg_last_error(NULL) says so, and nothing stays allocated."""
    free0 = free_bytes(torch)
    failures = 0
    for after in range(0, 16):
        B.inject_alloc_failure(after)
        try:
            with B.Lattice(**CFG) as lat:
                lat.init()
            break  # `after` is past the create's allocations: it succeeded
        except B.IlgError as e:
            assert e.status == B.ILG_E_OOM, e
            assert "out of memory" in str(e), e
            failures += 1
        finally:
            B.inject_alloc_failure(-1)
    assert failures >= 5  # two state buffers, tables, the overflow word, the sums
    assert abs(free_bytes(torch) - free0) < (16 << 20)


def test_context_works_after_injected_failure(B, torch):
    B.inject_alloc_failure(0)
    with pytest.raises(B.IlgError):
        B.Lattice(**CFG)
    B.inject_alloc_failure(-1)
    with B.Lattice(**CFG) as lat:
        lat.init()
        lat.step(3)
        got, t = lat.get_state()
    ref = O.Lattice(**CFG)
    assert t == 3 and np.array_equal(got, ref.run(ref.init(), 0, 3))


def test_no_leak_over_create_destroy_cycles(B, torch):
    """Creates that fail half way and creates that succeed, many times over: device
    memory comes back each time."""
    free0 = free_bytes(torch)
    for k in range(30):
        if k % 2:
            B.inject_alloc_failure(k % 5)
            with pytest.raises(B.IlgError):
                B.Lattice(**CFG)
            B.inject_alloc_failure(-1)
        else:
            with B.Lattice(**CFG) as lat:
                lat.init()
    assert abs(free_bytes(torch) - free0) < (16 << 20)


def test_batch_and_server_and_comparator_creates_report_oom(B, torch):
    free0 = free_bytes(torch)
    reps = [dict(lattice=1, Lx=64 + 8 * i, n0=10.0, omega_eff=1.5, seed=3, replica=i) for i in range(4)]
    for after in (0, 2, 4):
        B.inject_alloc_failure(after)
        try:
            with pytest.raises(B.IlgError) as e:
                B.Batch(reps)
            assert e.value.status == B.ILG_E_OOM
        finally:
            B.inject_alloc_failure(-1)
    for after in (0, 1, 3):
        B.inject_alloc_failure(after)
        try:
            with pytest.raises(B.IlgError) as e:
                B.Server(3, 64 << 20, max_slots=4, quantum=4)
            assert e.value.status == B.ILG_E_OOM
        finally:
            B.inject_alloc_failure(-1)
    B.inject_alloc_failure(0)
    try:
        with pytest.raises(B.IlgError) as e:
            B.LB(lattice=2, Lx=64, Ly=64, omega_j=1.5, omega=0.5)
        assert e.value.status == B.ILG_E_OOM
    finally:
        B.inject_alloc_failure(-1)
    # and each works afterwards
    with B.Batch(reps) as bat:
        bat.init()
        bat.run(3)
    with B.Server(3, 64 << 20, max_slots=4, quantum=4) as srv:
        srv.submit(0, steps=5, lattice=2, Lx=32, Ly=32, n0=6.0, omega_eff=1.5, seed=3, replica=0)
        srv.wait_idle(60)
        assert srv.poll()[0]["status"] == B.ILG_OK
    assert abs(free_bytes(torch) - free0) < (16 << 20)


def test_injection_off_by_default(B, torch):
    """Without an injected failure the countdown is off: many creates succeed."""
    for _ in range(5):
        with B.Lattice(**CFG):
            pass
