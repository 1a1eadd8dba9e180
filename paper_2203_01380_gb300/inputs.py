"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the method: it only draws random numbers
(numpy PCG64, fixed seeds) for initial states handed to ``ilg_set_state``,
parameters of replica ensembles and request streams.  Both the CUDA path and
the oracle take these inputs unchanged.

Workloads (the paper uses no dataset; every input is generated):
  ring_d1q3      D1Q3 ring L=256, per-velocity Poisson mean 30, density sine
                 amplitude 10 at k = 2 pi / L, omega_eff 1.5, 2000 steps, seed 1
  sweep_d2q5     D2Q5 1024^2, mean 50 per velocity, sine amplitude 20 at
                 k = (2 pi / 1024, 0), omega_eff in {0.5, 1.0, 1.5, 1.9},
                 1000 steps each, seed 2, replica = sweep index
  large_d2q5     D2Q5 16384^2, uniform mean 10 per velocity, omega_eff 1.8,
                 500 steps, seed 3, structure factor for axis modes 1..64
  batch_d1q3     4096 D1Q3 rings, L log-uniform in [64, 8192], mean occupation
                 uniform in [5, 200], omega_eff uniform in [0.2, 1.95],
                 5000 steps, seed 4, replica = index
  serve_d2q5     Poisson arrivals (200 / s) of D2Q5 requests, side log-uniform
                 in [64, 2048], steps log-uniform in [100, 10000], mean
                 occupation uniform in [5, 100], omega_eff 1.5, seed 5
  large_d2q9     D2Q9 16384^2 (weights 4/9, 1/9, 1/36), mean 10 per velocity,
                 omega_eff 1.8, 100 steps, seed 3
  lb_d2q5        lattice Boltzmann comparator on 16384^2 (D2Q5), initial f the
                 sweep's Poisson means (50 per velocity, sine amplitude 20 along
                 x), rates of the gas with omega_eff 1.8, 200 steps
  ensemble_d1q3  512 replicas of one D1Q3 ring L=320 (Sec. V: wavelength 320),
                 mean density 100 with sine amplitude 100, omega_eff 1.5, seed 6
"""
from __future__ import annotations

import numpy as np

D1Q3, D2Q5, D2Q9 = 1, 2, 3

RING_D1Q3 = dict(lattice=D1Q3, Lx=256, Ly=1, n0=30.0, amp=10.0, mode_mx=1, mode_my=0,
                 init_weighted=0, omega_eff=1.5, theta=1.0 / 3.0, seed=1, replica=0, steps=2000)
SWEEP_D2Q5 = [dict(lattice=D2Q5, Lx=1024, Ly=1024, n0=50.0, amp=20.0, mode_mx=1, mode_my=0,
                   init_weighted=0, omega_eff=w, theta=1.0 / 3.0, seed=2, replica=i, steps=1000)
              for i, w in enumerate((0.5, 1.0, 1.5, 1.9))]
LARGE_D2Q5 = dict(lattice=D2Q5, Lx=16384, Ly=16384, n0=10.0, amp=0.0, mode_mx=0, mode_my=0,
                  init_weighted=0, omega_eff=1.8, theta=1.0 / 3.0, seed=3, replica=0, steps=500)
LARGE_MODES = [(m, 0) for m in range(1, 65)]
LARGE_D2Q9 = dict(lattice=3, Lx=16384, Ly=16384, n0=10.0, amp=0.0, mode_mx=0, mode_my=0,
                  init_weighted=0, omega_eff=1.8, theta=1.0 / 3.0, seed=3, replica=0, steps=100)
LB_D2Q5 = dict(lattice=D2Q5, Lx=16384, Ly=16384, n0=50.0, amp=20.0, mode_mx=1, mode_my=0,
               init_weighted=0, omega_eff=1.8, theta=1.0 / 3.0, steps=200)
ENSEMBLE_D1Q3 = dict(lattice=D1Q3, Lx=320, Ly=1, n0=100.0 / 3.0, amp=100.0, mode_mx=1, mode_my=0,
                     init_weighted=1, omega_eff=1.5, theta=1.0 / 3.0, seed=6, replicas=512, steps=2000)


def scaled(cfg: dict, **over) -> dict:
    """A copy of a workload with some fields replaced (smaller sizes, fewer steps)."""
    c = dict(cfg)
    c.update(over)
    return c


def random_state(Q: int, Ly: int, Lx: int, mean: float, seed: int, hot: int = 0,
                 hot_value: int = 0) -> np.ndarray:
    """Poisson(mean) occupations, shape (Q, Ly, Lx) uint16; optionally `hot`
    randomly placed entries set to `hot_value` (large occupations)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = rng.poisson(mean, size=(Q, Ly, Lx))
    if hot:
        flat = s.reshape(-1)
        idx = rng.choice(flat.size, size=hot, replace=False)
        flat[idx] = hot_value
    return np.clip(s, 0, 65535).astype(np.uint16)


def batch_replicas(n: int = 4096, seed: int = 4, L_min: int = 64, L_max: int = 8192,
                   n0_range=(5.0, 200.0), omega_range=(0.2, 1.95)) -> list[dict]:
    """Parameters of n independent D1Q3 rings (replica index = position)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = np.exp(rng.uniform(np.log(L_min), np.log(L_max), size=n)).astype(np.int64)
    n0 = rng.uniform(*n0_range, size=n)
    om = rng.uniform(*omega_range, size=n)
    return [dict(lattice=D1Q3, Lx=int(L[i]), Ly=1, n0=float(n0[i]), amp=0.0, mode_mx=0,
                 mode_my=0, init_weighted=0, omega_eff=float(om[i]), theta=1.0 / 3.0,
                 seed=seed, replica=i) for i in range(n)]


def serve_requests(n: int, seed: int = 5, rate: float = 200.0, side_range=(64, 2048),
                   steps_range=(100, 10000), n0_range=(5.0, 100.0),
                   omega_eff: float = 1.5) -> list[dict]:
    """A Poisson arrival stream of D2Q5 requests (arrival times in seconds)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrive = np.cumsum(gaps)
    side = np.exp(rng.uniform(np.log(side_range[0]), np.log(side_range[1]), size=n)).astype(np.int64)
    steps = np.exp(rng.uniform(np.log(steps_range[0]), np.log(steps_range[1]), size=n)).astype(np.int64)
    n0 = rng.uniform(*n0_range, size=n)
    return [dict(arrive=float(arrive[i]), lattice=D2Q5, Lx=int(side[i]), Ly=int(side[i]),
                 n0=float(n0[i]), amp=0.0, mode_mx=0, mode_my=0, init_weighted=0,
                 omega_eff=omega_eff, theta=1.0 / 3.0, seed=seed, replica=i,
                 steps=int(steps[i])) for i in range(n)]
