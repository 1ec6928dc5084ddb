"""The ideal-gas reservoir relation of Sec. III.A in the library
(regc_mu_of_pressure, regc_pressure_of_mu) against the oracle's, and a
consistency check of the B mass the workloads infer from the paper's state
point (200 K, 2.03e-17 atm), which Sec. III.A places at the corner state
(200 K, -0.9 eV).  Both entry points are host code of the library: no GPU is
needed."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mbar as OM
from paper_1908_11118_gb300 import build as B
from paper_1908_11118_gb300 import mu_of_pressure, pressure_of_mu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_pressure_relation_matches_oracle_and_round_trips():
    rng = np.random.default_rng(0)
    kT = rng.uniform(0.01, 2.0, 50)
    p = 10.0 ** rng.uniform(-25, 0, 50)
    for lam0 in (1.0, W.thermal_lambda0(W.PAPER_B_MASS_AMU)):
        mu = mu_of_pressure(kT, p, lam0)
        np.testing.assert_allclose(mu, OM.mu_from_pressure(kT, p, lam0), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(pressure_of_mu(kT, mu, lam0), p, rtol=1e-12)
    with pytest.raises(Exception):
        mu_of_pressure([1.0], [-1.0], 1.0)


def test_paper_state_point_consistency():
    """The mass is inferred from the first state point, so reproducing it is a
    consistency check, not a pin: here the mass is derived again in SI units
    from Lambda = h / sqrt(2 pi m kT) and p Lambda^3 = kT exp(mu / kT), and the
    library then maps the paper's second printed state point (600 K,
    8.89e-2 atm) to mu = -0.980 eV with that mass (the paper prints no mu for
    it; three digits of its pressure fix mu to about 1e-4 eV)."""
    k_b = 1.380649e-23                              # J / K (SI, exact)
    T, p, mu = 200.0, 2.03e-17 * 101325.0, -0.9 * W.EV_J
    lam = (k_b * T * math.exp(mu / (k_b * T)) / p) ** (1.0 / 3.0)
    m = W.PLANCK_J_S ** 2 / (2.0 * math.pi * k_b * T * lam * lam) / W.AMU_KG
    assert abs(m - W.PAPER_B_MASS_AMU) < 1e-6 * m
    lam0 = W.thermal_lambda0(W.PAPER_B_MASS_AMU)
    mu = mu_of_pressure(W.K_B_EV * np.array([200.0, 600.0]), np.array([2.03e-17, 8.89e-2]) * W.ATM_EV_PER_A3, lam0)
    assert abs(mu[0] + 0.9) < 1e-9
    assert abs(mu[1] + 0.980) < 5e-4
