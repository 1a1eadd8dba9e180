"""Ensemble statistics of batched rings (ilg_batch_ensemble): per-ring complex
mode amplitudes against the oracle, the on-device reduction against a plain
numpy reduction of the same record, and the statistics against their exact
values for Poisson starts (product-Poisson propagation through the lattice
Boltzmann map of Sec. IV, computed by the oracle)."""
import math

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


def numpy_stats(rec):
    a = rec[..., 0] + 1j * rec[..., 1]
    n = a.shape[0]
    m = a.mean(axis=0)
    d = a - m[None, :]
    cov = (d * np.conj(d[:, :1])).sum(axis=0) / (n - 1)
    return dict(mean_re=m.real, mean_im=m.imag, var_re=(d.real ** 2).sum(0) / (n - 1),
                var_im=(d.imag ** 2).sum(0) / (n - 1), cov_re=cov.real, cov_im=cov.imag)


@pytest.mark.parametrize("mode", [1, -3])
def test_record_matches_oracle_and_reduction_matches_numpy(B, mode):
    L, T = 40, 12
    reps = [dict(lattice=1, Lx=L, n0=25.0, amp=20.0, mode_mx=1, init_weighted=1, omega_eff=w, seed=12, replica=i)
            for i, w in enumerate([1.5, 1.5, 0.8, 1.9, 1.0, 1.5])]
    with B.Batch(reps) as bat:
        bat.init()
        st = bat.ensemble(T, mode=mode, record=True)
    rec = st["record"]
    for i, r in enumerate(reps):
        lat = O.Lattice(**r)
        s = lat.init()
        for t in range(T + 1):
            _, _, _, res = lat.observables(s, [(mode, 0)])
            tol = 1e-12 * res[0]["scale"] + 1e-12
            assert abs(rec[i, t, 0] - res[0]["re"]) <= tol, (i, t)
            assert abs(rec[i, t, 1] - res[0]["im"]) <= tol, (i, t)
            if t < T:
                s = lat.step(s, t)
    ref = numpy_stats(rec)
    for k in B.Batch.ENSEMBLE_ROWS:
        scale = np.abs(ref[k]).max() + 1.0
        assert np.abs(st[k] - ref[k]).max() <= 1e-12 * scale, k


def test_statistics_are_deterministic(B):
    reps = [dict(lattice=1, Lx=64, n0=10.0, amp=5.0, mode_mx=1, omega_eff=1.3, seed=2, replica=i) for i in range(300)]
    out = []
    for _ in range(2):
        with B.Batch(reps) as bat:
            bat.init()
            out.append(bat.ensemble(50, mode=1))
    for k in B.Batch.ENSEMBLE_ROWS:
        assert np.array_equal(out[0][k], out[1][k]), k


def test_statistics_match_exact_values(B):
    """4096 replicas of the ensemble ring (L = 320, Sec. V's wavelength) for 300 steps:
    mean amplitude (the Fig. 1 observable), variances and the dynamic correlation
    within six standard errors of their exact values at every t."""
    cfg = {k: v for k, v in inputs.ENSEMBLE_D1Q3.items() if k not in ("replicas", "steps")}
    R, T, mode = 4096, 300, 1
    reps = [dict(cfg, replica=r) for r in range(R)]
    with B.Batch(reps) as bat:
        bat.init()
        st = bat.ensemble(T, mode=mode)
    oj, om = OL.rates_from_omega_eff(cfg["omega_eff"])
    lb = OL.LB(1, cfg["Lx"], omega_j=oj, omega=om, theta=cfg["theta"])
    f0 = lb.init_mean(n0=cfg["n0"], amp=cfg["amp"], mode_mx=cfg["mode_mx"], init_weighted=cfg["init_weighted"])
    pred = OL.ensemble_prediction(lb, f0, mode, T)
    tot0 = pred["var_re"][0] + pred["var_im"][0]
    for t in range(T + 1):
        assert abs(st["mean_re"][t] - pred["mean_re"][t]) < 6 * math.sqrt(pred["var_re"][t] / R), t
        assert abs(st["mean_im"][t] - pred["mean_im"][t]) < 6 * math.sqrt(pred["var_im"][t] / R), t
        assert abs(st["var_re"][t] / pred["var_re"][t] - 1) < 6 * math.sqrt(2 / R) + 0.01, t
        assert abs(st["var_im"][t] / pred["var_im"][t] - 1) < 6 * math.sqrt(2 / R) + 0.01, t
        se = math.sqrt((pred["var_re"][t] + pred["var_im"][t]) * tot0 / R)
        assert abs(st["cov_re"][t] - pred["cov_re"][t]) < 6 * se, t
        assert abs(st["cov_im"][t] - pred["cov_im"][t]) < 6 * se, t
    # the mean amplitude decays (the signal of Fig. 1) by many standard errors, so a
    # wrong decay rate would fail the comparison above
    assert pred["mean_im"][0] - pred["mean_im"][T] > 20 * math.sqrt(pred["var_im"][T] / R)


def test_ensemble_errors(B):
    mixed = [dict(lattice=1, Lx=L, seed=1, replica=i) for i, L in enumerate([32, 33])]
    with B.Batch(mixed) as bat:
        bat.init()
        with pytest.raises(B.IlgError):
            bat.ensemble(4)
    with B.Batch([dict(lattice=1, Lx=32, seed=1)]) as bat:
        bat.init()
        with pytest.raises(B.IlgError):
            bat.ensemble(4)
    with B.Batch([dict(lattice=1, Lx=32, seed=1, replica=i) for i in range(3)]) as bat:
        bat.init()
        with pytest.raises(B.IlgError):
            bat.ensemble(4, mode=64)


def test_ensemble_zero_steps_and_particle_sampler(B):
    """T = 0 gives the statistics of the initial states alone; rings with the particle
    sampler give records equal to the oracle's."""
    L = 24
    reps = [dict(lattice=1, Lx=L, n0=12.0, amp=8.0, mode_mx=1, omega_eff=1.3, seed=3, replica=i, sampler=1)
            for i in range(5)]
    with B.Batch(reps) as bat:
        bat.init()
        st0 = bat.ensemble(0, mode=1, record=True)
        assert st0["record"].shape == (5, 1, 2)
        st = bat.ensemble(6, mode=1, record=True)
    for i, r in enumerate(reps):
        lat = O.Lattice(**r)
        s = lat.init()
        _, _, _, res = lat.observables(s, [(1, 0)])
        assert abs(st0["record"][i, 0, 1] - res[0]["im"]) <= 1e-12 * res[0]["scale"] + 1e-12
        for t in range(6):
            s = lat.step(s, t)
        _, _, _, res = lat.observables(s, [(1, 0)])
        assert abs(st["record"][i, 6, 1] - res[0]["im"]) <= 1e-12 * res[0]["scale"] + 1e-12
