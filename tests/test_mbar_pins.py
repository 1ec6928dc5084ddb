"""Pins of the MBAR oracle (Sec. II.B) against closed forms.

* One state: MBAR reduces to the plain sample average.
* Ideal gas with exact expected counts: the grand-canonical partition function
  is Xi_s = sum_{N <= Nmax} lambda_s^N / N!, lambda_s = V exp(beta_s mu_s) / Lambda_s^3.
  With histograms proportional to the exact truncated-Poisson probabilities of
  several (T, mu) states, MBAR must return f_s - f_0 = -ln(Xi_s / Xi_0), and
  reweighting to any other (T, mu) must return that state's truncated Poisson
  mean and probabilities.  This fails if the thermal-wavelength term of the
  reduced potential is dropped while the states differ in T.
* The pressure form mu(T, p) of Sec. III.A against the ideal-gas relation
  <N> = p V / kT (untruncated limit).
"""
import math

import numpy as np
import pytest

from oracle import mbar


def _poisson(lam, nmax):
    n = np.arange(nmax + 1)
    lp = n * math.log(lam) - np.array([math.lgamma(k + 1) for k in n])
    return lp


def _ideal_setup(nmax=40, V=50.0):
    kT = np.array([0.7, 0.7, 0.7, 1.1, 1.1, 1.1, 1.6, 1.6, 1.6])
    mu = np.array([-4.0, -3.0, -2.5, -4.0, -3.2, -2.6, -4.5, -3.8, -3.0])
    lam = V * np.exp(mu / kT) * kT ** 1.5
    omega = np.array([1000.0, 2000.0, 1500.0, 800.0, 1200.0, 900.0, 1000.0, 1000.0, 3000.0])
    H = np.zeros(nmax + 1)
    lnxi = np.zeros(len(kT))
    for s in range(len(kT)):
        lp = _poisson(lam[s], nmax)
        lnxi[s] = mbar.lse(lp)
        H += omega[s] * np.exp(lp - lnxi[s])
    return kT, mu, lam, omega, H, lnxi, V


def test_single_state_is_sample_mean():
    rng = np.random.default_rng(0)
    N = rng.integers(0, 10, 500).astype(float)
    E = rng.normal(-5, 2, 500)
    f, D, _, ok = mbar.solve([1.2], [-3.0], 1.0, [500], N, E, np.ones(500))
    assert ok and f[0] == 0.0
    n_mean, p_N, _ = mbar.query([1.2], [-3.0], 1.0, N, E, np.ones(500), D, 10)
    assert n_mean[0] == pytest.approx(N.mean(), rel=1e-12)
    assert p_N[0] @ np.arange(11) == pytest.approx(N.mean(), rel=1e-12)


def test_ideal_gas_free_energies_exact():
    nmax = 40
    kT, mu, lam, omega, H, lnxi, V = _ideal_setup(nmax)
    N_b = np.arange(nmax + 1, dtype=float)
    E_b = np.zeros(nmax + 1)
    # the reduced potential is relative to the measure V^N/N!: put V into the bins
    # by shifting mu (ln V per particle at each beta), i.e. query the same thing
    f, D, it, ok = mbar.solve(kT, mu + kT * math.log(V), 1.0, omega, N_b, E_b, H, tol=1e-12)
    assert ok
    np.testing.assert_allclose(f, -(lnxi - lnxi[0]), atol=1e-9)


def test_exact_free_energies_are_the_fixed_point_of_one_map():
    """Started at the closed-form f, one map of the plain iteration stays
    there; started elsewhere, the iteration returns to it."""
    nmax = 40
    kT, mu, lam, omega, H, lnxi, V = _ideal_setup(nmax)
    N_b = np.arange(nmax + 1, dtype=float)
    E_b = np.zeros(nmax + 1)
    exact = -(lnxi - lnxi[0])
    f1, _, it, _ = mbar.solve(kT, mu + kT * math.log(V), 1.0, omega, N_b, E_b, H, max_iter=1, f0=exact)
    assert it == 1
    np.testing.assert_allclose(f1, exact, atol=1e-12)
    start = exact + np.linspace(-3.0, 3.0, len(exact))
    f2, _, _, ok = mbar.solve(kT, mu + kT * math.log(V), 1.0, omega, N_b, E_b, H, tol=1e-13, f0=start)
    assert ok
    np.testing.assert_allclose(f2, exact, atol=1e-9)


def test_ideal_gas_reweighting_off_grid():
    nmax = 40
    kT, mu, lam, omega, H, lnxi, V = _ideal_setup(nmax)
    N_b = np.arange(nmax + 1, dtype=float)
    E_b = np.zeros(nmax + 1)
    f, D, it, ok = mbar.solve(kT, mu + kT * math.log(V), 1.0, omega, N_b, E_b, H, tol=1e-12)
    kq = np.array([0.8, 1.0, 1.3, 1.5])
    mq = np.array([-3.5, -3.1, -3.6, -3.3])
    n_mean, p_N, _ = mbar.query(kq, mq + kq * math.log(V), 1.0, N_b, E_b, H, D, nmax)
    for q in range(len(kq)):
        lp = _poisson(V * math.exp(mq[q] / kq[q]) * kq[q] ** 1.5, nmax)
        pr = np.exp(lp - mbar.lse(lp))
        assert n_mean[q] == pytest.approx(pr @ N_b, rel=1e-9)
        np.testing.assert_allclose(p_N[q], pr, atol=1e-11)


def test_dropping_the_wavelength_term_is_detected():
    nmax = 40
    kT, mu, lam, omega, H, lnxi, V = _ideal_setup(nmax)
    N_b = np.arange(nmax + 1, dtype=float)
    E_b = np.zeros(nmax + 1)
    wrong = lambda kT_, mu_, lam0, N, E: (np.asarray(E)[None, :] - np.asarray(mu_)[:, None] * np.asarray(N)[None, :]) / np.asarray(kT_)[:, None]
    orig = mbar.reduced_potential
    try:
        mbar.reduced_potential = wrong
        f, D, it, ok = mbar.solve(kT, mu + kT * math.log(V), 1.0, omega, N_b, E_b, H, tol=1e-12)
    finally:
        mbar.reduced_potential = orig
    assert np.max(np.abs(f + (lnxi - lnxi[0]))) > 1e-2


def test_pressure_relation_ideal_gas():
    # untruncated ideal gas: <N> = lambda = V exp(beta mu) / Lambda^3 = p V / kT
    kT = np.array([0.6, 1.0, 1.5])
    p = np.array([1e-3, 2e-2, 5e-1])
    mu = mbar.mu_from_pressure(kT, p, 1.0)
    lam = 100.0 * np.exp(mu / kT) / (1.0 / np.sqrt(kT)) ** 3
    np.testing.assert_allclose(lam, p * 100.0 / kT, rtol=1e-12)


def _ideal2_setup(nmax=20, V=50.0, lam0_2=0.7):
    """Two ideal species (B: lambda0 1, C: lambda0_2) on six (kT, mu_B, mu_C)
    states, histograms proportional to the exact probabilities of the product
    of two Poisson laws truncated to N_B + N_C <= nmax."""
    kT = np.array([0.7, 0.7, 1.1, 1.1, 1.6, 1.6])
    mu = np.array([-4.0, -3.2, -3.6, -3.0, -4.2, -3.4])
    mu2 = np.array([-3.6, -4.1, -3.2, -3.9, -3.5, -4.4])
    omega = np.array([1000.0, 2000.0, 1500.0, 800.0, 1200.0, 900.0])
    a = np.arange(nmax + 1)
    NB, NC = np.meshgrid(a, a, indexing="ij")
    keep = NB + NC <= nmax
    NB, NC = NB[keep].astype(float), NC[keep].astype(float)
    lg = np.array([math.lgamma(k + 1) for k in range(nmax + 1)])
    H = np.zeros(len(NB))
    lnxi = np.zeros(len(kT))
    for s in range(len(kT)):
        lb = math.log(V) + mu[s] / kT[s] + 1.5 * math.log(kT[s])
        lc = math.log(V) + mu2[s] / kT[s] - 3 * math.log(lam0_2) + 1.5 * math.log(kT[s])
        lp = NB * lb + NC * lc - lg[NB.astype(int)] - lg[NC.astype(int)]
        lnxi[s] = mbar.lse(lp)
        H += omega[s] * np.exp(lp - lnxi[s])
    return kT, mu, mu2, omega, NB, NC, H, lnxi, V, lam0_2


def test_two_species_ideal_gas_free_energies_and_reweighting():
    """With two species the partition function is the truncated double sum
    Xi_s = sum_{a + b <= nmax} lambda_B^a / a! lambda_C^b / b!: MBAR must give
    f_s - f_0 = -ln(Xi_s / Xi_0), and reweighting to other (kT, mu_B, mu_C)
    the exact truncated means of both counts."""
    nmax = 20
    kT, mu, mu2, omega, NB, NC, H, lnxi, V, l2 = _ideal2_setup(nmax)
    E = np.zeros(len(NB))
    lnV = math.log(V)
    f, D, it, ok = mbar.solve(kT, mu + kT * lnV, 1.0, omega, NB, E, H, tol=1e-12,
                              mu2_s=mu2 + kT * lnV, N2_b=NC, lambda0_2=l2)
    assert ok
    np.testing.assert_allclose(f, -(lnxi - lnxi[0]), atol=1e-9)
    kq, mq, m2q = np.array([0.8, 1.3]), np.array([-3.5, -3.3]), np.array([-3.8, -3.6])
    nb, nc, pB, pC, _ = mbar.query2(kq, mq + kq * lnV, m2q + kq * lnV, 1.0, l2, NB, NC, E, H, D, nmax)
    lg = np.array([math.lgamma(k + 1) for k in range(nmax + 1)])
    for q in range(len(kq)):
        lb = lnV + mq[q] / kq[q] + 1.5 * math.log(kq[q])
        lc = lnV + m2q[q] / kq[q] - 3 * math.log(l2) + 1.5 * math.log(kq[q])
        lp = NB * lb + NC * lc - lg[NB.astype(int)] - lg[NC.astype(int)]
        w = np.exp(lp - mbar.lse(lp))
        assert nb[q] == pytest.approx(w @ NB, rel=1e-9)
        assert nc[q] == pytest.approx(w @ NC, rel=1e-9)
        assert pB[q].sum() == pytest.approx(1.0, abs=1e-12)
    # planted: the second species' chemical potential left out
    f_bad, _, _, _ = mbar.solve(kT, mu + kT * lnV, 1.0, omega, NB, E, H, tol=1e-12,
                                mu2_s=np.zeros_like(mu2), N2_b=NC, lambda0_2=l2)
    assert np.max(np.abs(f_bad + (lnxi - lnxi[0]))) > 1e-2
