"""The paper's results reproduced on the GPU path (synthetic runs; the paper's own
data is not in its source).

* Sec. V, Fig. 1: D1Q3, L = 320, N^ave = 100, an ensemble of 500 runs per omega^j,
  the mean amplitude of the sine wave against the exact mean dynamics of Sec. IV and
  against A^th(t) = N^ave exp(-4 pi^2 D t / L^2) with D = theta (1/omega^j - 1/2).
* The D2Q5 sweep (1024^2, mean 50 + density sine of amplitude 20, 1000 steps,
  omega_eff in {0.5, 1.0, 1.5, 1.9}): the measured amplitude follows the exact mean
  dynamics; where the decay is resolved, its rate matches D k^2.
"""
import numpy as np
import pytest

from paper_2203_01380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import binding
    return binding


def lb_amplitudes(Q, w, flip, omega_star, f0, steps, L, every=1):
    """Exact mean dynamics (Sec. IV) of a sine mode on an L-periodic axis; f0 shape (Q, L)
    along that axis (the other axis uniform, so D2Q5's +-y planes do not move it)."""
    opp = [0, 2, 1] if Q == 3 else [0, 2, 1, 4, 3]
    w = np.asarray(w)[:, None]
    f = f0.copy()
    s = np.sin(2 * np.pi * np.arange(L) / L)
    out = []
    for t in range(1, steps + 1):
        g = f[opp] if flip else f
        rho = g.sum(axis=0)
        post = g + omega_star * (w * rho[None, :] - g)
        f = post.copy()
        f[1] = np.roll(post[1], 1)
        f[2] = np.roll(post[2], -1)
        if t % every == 0:
            out.append(float((s * f.sum(axis=0)).sum() / (L / 2)))
    return np.array(out)


@pytest.mark.parametrize("omega_j", [0.5, 1.0, 1.5, 1.9])
def test_fig1_ensemble_amplitude(B, omega_j):
    L, n_ave, runs, T = 320, 100.0, 500, 1500
    theta = 1.0 / 3.0
    reps = [dict(lattice=1, Lx=L, n0=n_ave / 3.0, amp=n_ave, mode_mx=1, init_weighted=1,
                 omega_eff=omega_j, theta=theta, seed=2022, replica=i) for i in range(runs)]
    with B.Batch(reps) as bat:
        bat.init()
        rec = bat.run(T, record_mode=1)
    mean = rec.mean(axis=0)
    sem = rec.std(axis=0, ddof=1) / np.sqrt(runs)
    w = [1 - theta, theta / 2, theta / 2]
    flip = omega_j > 1.0
    om = 2.0 - omega_j if flip else omega_j
    x = np.arange(L)
    rho0 = n_ave * (1 + np.sin(2 * np.pi * x / L))
    f0 = np.stack([wi * rho0 for wi in w])
    exact = lb_amplitudes(3, w, flip, om, f0, T, L)
    idx = np.linspace(0, T - 1, 16).astype(int)
    assert np.all(np.abs(mean[idx] - exact[idx]) < 5 * sem[idx] + 1e-9), (mean[idx], exact[idx])
    # the paper's closed form (continuum limit of Sec. IV): a few percent of A^th
    D = theta * (1.0 / omega_j - 0.5)
    t = np.arange(1, T + 1)
    Ath = n_ave * np.exp(-4 * np.pi ** 2 * D * t / L ** 2)
    assert np.all(np.abs(mean[idx] - Ath[idx]) < 0.03 * n_ave + 5 * sem[idx])


def test_d2q5_sweep_decay(B):
    every = 100
    for c in inputs.SWEEP_D2Q5:
        cfg = {k: v for k, v in c.items() if k != "steps"}
        T, L = c["steps"], cfg["Lx"]
        amps = []
        with B.Lattice(**cfg) as lat:
            lat.init()
            for _ in range(T // every):
                lat.step(every)
                amps.append(lat.observables([(1, 0)])["amp"][0])
        amps = np.array(amps)
        theta = cfg["theta"]
        w = [1 - 2 * theta] + [theta / 2] * 4
        flip = cfg["omega_eff"] > 1.0
        om = 2.0 - cfg["omega_eff"] if flip else cfg["omega_eff"]
        lam = cfg["n0"] + cfg["amp"] * np.sin(2 * np.pi * np.arange(L) / L) / 5
        f0 = np.stack([lam] * 5)
        exact = lb_amplitudes(5, w, flip, om, f0, T, L, every=every)
        sigma = np.sqrt(5 * cfg["n0"] / (L * L / 2))      # product-Poisson noise of A^LG
        assert np.all(np.abs(amps - exact) < 6 * sigma), (cfg["omega_eff"], amps, exact)
        if cfg["omega_eff"] <= 1.0:                      # decay resolved over 1000 steps
            D = theta * (1.0 / cfg["omega_eff"] - 0.5)
            k = 2 * np.pi / L
            t = every * np.arange(1, len(amps) + 1)
            rate = -np.polyfit(t, np.log(amps), 1)[0]
            assert abs(rate / (D * k * k) - 1) < 0.25, (cfg["omega_eff"], rate, D * k * k)
