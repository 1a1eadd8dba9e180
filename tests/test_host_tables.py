"""The library's host-side table builders against the oracle's, on the CPU.

The integer CDF rows, the 64-column alias tables and the Poisson tables the kernels
read are built on the host by libilg.so's own code (no GPU involved); the oracle
builds the same tables independently.  They must agree bit for bit."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def B():
    from paper_2203_01380_gb300 import build as b
    b.build()
    from paper_2203_01380_gb300 import binding
    return binding


PS = [1, 17, O.quantise(1e-6), O.quantise(0.05), O.quantise(0.2), O.quantise(1.0 / 3.0), 1 << 31,
      O.quantise(2.0 / 3.0), O.quantise(0.95), (1 << 32) - 17, (1 << 32) - 1]


@pytest.mark.parametrize("P", PS)
def test_binomial_and_alias_tables(B, P):
    assert np.array_equal(B.binomial_table(P), O.binomial_table(P))
    thr, al = B.alias_table(P)
    othr, oal = O.alias_table(P)
    assert np.array_equal(thr, othr) and np.array_equal(al, oal.astype(np.uint32))


@pytest.mark.parametrize("lam", [0.0, 1e-9, 0.25, 3.0, 10.0, 33.33, 100.0, 450.5, 700.0])
def test_poisson_tables(B, lam):
    assert np.array_equal(B.poisson_table(lam), O.poisson_table(lam))


def test_table_arguments_are_checked(B):
    for P in (0, 1 << 32):
        with pytest.raises(B.IlgError):
            B.alias_table(P)
        with pytest.raises(B.IlgError):
            B.binomial_table(P)
    with pytest.raises(B.IlgError):
        B.poisson_table(700.5)
    with pytest.raises(B.IlgError):
        B.poisson_table(-1.0)


@pytest.mark.parametrize("omega_eff", [0.2, 0.5, 1.0, 1.0000001, 1.5, 1.8, 2.0])
def test_lb_rates_match_the_oracle(B, omega_eff):
    """ilg_lb_rates (host only) against the oracle's mapping of Sec. IV, Eq. omegaj."""
    from oracle import lb as L
    assert B.lb_rates(omega_eff) == tuple(L.rates_from_omega_eff(omega_eff))


@pytest.mark.parametrize("omega_eff", [0.0, -1.0, 2.5, float("nan")])
def test_lb_rates_refuse_bad_parameters(B, omega_eff):
    with pytest.raises(B.IlgError):
        B.lb_rates(omega_eff)
