"""Serving loop (ilg_server_*): every request's result is the one it has alone,
whatever else runs beside it; admission waits for arena memory; waits are bounded."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu

SEED = 5


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


def requests(n, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.choice([8, 37, 64, 100, 128, 257, 512]))
        out.append(dict(lattice=2, Lx=side, Ly=side if i % 3 else side + 5, n0=float(rng.uniform(5, 80)),
                        amp=0.0, omega_eff=float(rng.choice([0.6, 1.0, 1.5, 1.9])), seed=SEED, replica=1000 + i,
                        steps=int(rng.integers(1, 90))))
    return out


def alone(B, r):
    cfg = {k: v for k, v in r.items() if k != "steps"}
    with B.Lattice(**cfg) as lat:
        lat.init()
        lat.step(r["steps"])
        s, t = lat.get_state()
        obs = lat.observables([(1, 0)])
    return s, t, obs


def check(B, reqs, results):
    by_id = {res["id"]: res for res in results}
    assert set(by_id) == {1000 + i for i in range(len(reqs))}
    for i, r in enumerate(reqs):
        res = by_id[1000 + i]
        s, t, obs = alone(B, r)
        assert res["status"] == 0 and res["t"] == t == r["steps"]
        assert np.array_equal(res["state"], s), i
        assert res["mass"] == obs["mass"]
        assert res["amp"] == obs["amp"][0] and res["Sk"] == obs["Sk"][0]
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]


def test_mix_equals_alone(B):
    reqs = requests(14)
    with B.Server(SEED, 1 << 30, max_slots=64, quantum=16) as srv:
        for i, r in enumerate(reqs):
            srv.submit(1000 + i, want_state=True, **r)
        srv.wait_idle(300)
        results = srv.poll()
    check(B, reqs, results)


def test_late_arrivals_join_and_small_arena_queues(B):
    """An arena for about two of the largest requests: the rest wait for memory;
    a second wave arrives while the first runs."""
    reqs = requests(10, seed=8)
    big = max(2 * 5 * r["Lx"] * r["Ly"] * 2 for r in reqs)
    with B.Server(SEED, 2 * big + (4 << 20), max_slots=3, quantum=8) as srv:
        for i, r in enumerate(reqs[:5]):
            srv.submit(1000 + i, want_state=True, **r)
        time.sleep(0.05)
        for i, r in enumerate(reqs[5:], start=5):
            srv.submit(1000 + i, want_state=True, **r)
        srv.wait_idle(300)
        st = srv.stats()
        results = srv.poll()
    assert st["peak_resident"] <= 3
    check(B, reqs, results)


def test_small_request_matches_oracle(B):
    r = dict(lattice=2, Lx=24, Ly=19, n0=12.0, amp=6.0, mode_mx=1, omega_eff=1.7, seed=SEED, replica=77, steps=33)
    with B.Server(SEED, 64 << 20, max_slots=4, quantum=10) as srv:
        srv.submit(5, want_state=True, **r)
        srv.wait_idle(60)
        (res,) = srv.poll()
    ref = O.Lattice(**{k: v for k, v in r.items() if k != "steps"})
    assert np.array_equal(res["state"], ref.run(ref.init(), 0, r["steps"]))


def test_particle_sampler_requests_match_oracle(B):
    """Requests with the particle sampler served beside binomial-sampler requests."""
    base = dict(lattice=2, Lx=20, Ly=17, n0=9.0, amp=4.0, mode_mx=1, omega_eff=1.6, seed=SEED, steps=21)
    reqs = [dict(base, replica=300 + i, sampler=i % 2) for i in range(4)]
    with B.Server(SEED, 64 << 20, max_slots=4, quantum=8) as srv:
        for i, r in enumerate(reqs):
            srv.submit(i, want_state=True, **r)
        srv.wait_idle(60)
        res = {x["id"]: x for x in srv.poll()}
    for i, r in enumerate(reqs):
        ref = O.Lattice(**{k: v for k, v in r.items() if k != "steps"})
        assert np.array_equal(res[i]["state"], ref.run(ref.init(), 0, r["steps"])), i


def test_invalid_request_and_bounded_wait(B):
    with B.Server(SEED, 256 << 20, max_slots=4, quantum=4) as srv:
        with pytest.raises(B.IlgError):
            srv.submit(1, steps=5, lattice=2, Lx=16, Ly=16, seed=SEED + 1)      # wrong seed
        srv.submit(2, steps=5, lattice=2, Lx=16, Ly=16, n0=1.0, amp=30.0, mode_mx=1, seed=SEED)  # negative mean
        srv.submit(3, steps=60000, lattice=2, Lx=1024, Ly=1024, n0=10.0, seed=SEED)
        with pytest.raises(B.IlgError) as e:
            srv.wait_idle(0.05)
        assert e.value.status == B.ILG_E_TIMEOUT
        srv.wait_idle(600)
        res = {r["id"]: r for r in srv.poll()}
    assert res[2]["status"] == B.ILG_E_INVALID and res[3]["status"] == 0 and res[3]["t"] == 60000


def test_least_work_first_admission(B):
    """With one slot and least-work-first admission, the requests queued behind a
    long first request are admitted smallest first; results are unchanged."""
    reqs = requests(6, seed=13)
    blocker = dict(lattice=2, Lx=512, Ly=512, n0=10.0, omega_eff=1.5, seed=SEED, replica=999)
    with B.Server(SEED, 1 << 30, max_slots=1, quantum=8) as srv:
        srv.set_policy(True)
        srv.submit(999, steps=400, **blocker)
        for i, r in enumerate(reqs):
            srv.submit(1000 + i, want_state=True, **r)
        srv.wait_idle(300)
        results = [r for r in srv.poll() if r["id"] != 999]
    check(B, reqs, results)
    order = sorted(results, key=lambda r: r["t_admit"])
    work = [reqs[r["id"] - 1000]["Lx"] * reqs[r["id"] - 1000]["Ly"] * reqs[r["id"] - 1000]["steps"] for r in order]
    assert work == sorted(work)
