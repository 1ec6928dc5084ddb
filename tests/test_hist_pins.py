"""Pins of the oracle's pooled (N, E) histogram and of the binned MBAR that
reads it (Sec. II.B: the observations of every state are pooled into bins
b = (N_b, E_b) before Eq. normlizationconstant is solved), against facts that
do not come from the oracle itself.

* Ideal gas (eps = 0): every configuration has E = 0 exactly, so every
  observation lands in the single bin k0 = floor(-e_lo / e_bin), in the row of
  the walker's N: hNE[:, k0] is the N marginal summed over states and every
  other bin is empty.  A window that excludes 0 leaves hNE empty and counts
  every observation as out of range; an edge at exactly 0 puts E = 0 in the
  bin above it (bins are closed below, open above).
* Interacting LJ gas: the mean of the bin energies equals the exact mean
  energy (the unbinned moments) within the spread of the position of an energy
  inside its bin, e_bin / sqrt(12 n): a bin index one too high, or bins taken
  at their lower edge, shift it by e_bin or e_bin / 2.  The N marginal of
  hNE equals the exact N moments.
* Small box with Nmax = 2: binned MBAR at chemical potentials that were not
  sampled reproduces the brute-force <N> and <E> of those states.
* Configuration 1 (16 states, Nmax 32): binned MBAR against unbinned MBAR (every
  observation its own bin) over the same observations: the free energies agree
  within the binning error, and the planted mistakes move them far beyond it.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mbar as MB
from oracle import oracle as O
from test_oracle_pins import brute_force_small_box, small_box_problem


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def run_ideal(e_lo, e_bin, n_bins, mutation=0, sweeps=300):
    p = W.ideal_gas(W.fcc100_small(L=2, M=3, nmax=24)).replace(e_lo=e_lo, e_bin=e_bin, n_e_bins=n_bins)
    orc = O.Oracle(p, mutation=mutation)
    orc.run(sweeps, exchange_every=10)
    return p, orc


def ideal_single_bin_error(mutation=0):
    """Number of observations that are not where E = 0 must put them."""
    p, orc = run_ideal(-1.0, 0.25, 16, mutation)
    k0 = 4                                       # floor((0 - (-1)) / 0.25)
    off = orc.hNE.copy()
    off[:, k0] = 0
    wrong_row = np.abs(orc.hNE[:, k0] - orc.hN.sum(axis=0)).sum()
    return int(off.sum() + wrong_row + orc.e_out.sum())


def test_ideal_gas_observations_fill_one_bin():
    assert ideal_single_bin_error() == 0
    p, orc = run_ideal(-1.0, 0.25, 16)
    assert orc.omega.sum() == 300 * p.S
    # the N marginal itself is the truncated Poisson law (pinned elsewhere); here
    # only check it is not degenerate, so the row test above means something
    assert np.count_nonzero(orc.hNE[:, 4]) > 5


def test_ideal_gas_window_edges():
    # a window above 0: nothing binned, every observation out of range
    p, orc = run_ideal(0.5, 0.25, 16, sweeps=40)
    assert orc.hNE.sum() == 0
    assert np.array_equal(orc.e_out, orc.omega)
    # an edge exactly at 0: E = 0 belongs to the bin above the edge
    p, orc = run_ideal(0.0, 0.25, 16, sweeps=40)
    assert orc.hNE[:, 0].sum() == orc.omega.sum() and orc.hNE[:, 1:].sum() == 0
    # a window that ends exactly at 0 excludes it
    p, orc = run_ideal(-4.0, 0.25, 16, sweeps=40)
    assert orc.hNE.sum() == 0 and orc.e_out.sum() == orc.omega.sum()


def test_ideal_gas_planted_bin_mistake_caught():
    assert ideal_single_bin_error(mutation=8192) > 1000


def lj_binned_mean_z(mutation=0, centre=0.5, sweeps=600):
    """z-score of (mean bin energy - exact mean energy) over every observation
    of a 16-state LJ run, against the spread e_bin / sqrt(12 n) of the position
    of an energy inside its bin; also returns the largest N-moment mismatch."""
    p = W.fcc100_small().replace(e_bin=0.1, n_e_bins=int(round(32 * 13.0 / 0.1)))
    pos, n = W.initial_walkers(p, [8] * p.S, seed=4)
    orc = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    orc.run(100, exchange_every=10, hist=False)
    orc.run(sweeps, exchange_every=10)
    assert orc.e_out.sum() == 0
    Nb, Eb, Hb = MB.occupied_bins(orc.hNE, p.e_lo, p.e_bin, centre=centre)
    n_obs = Hb.sum()
    assert n_obs == orc.omega.sum()
    e_binned = (Hb @ Eb) / n_obs
    e_exact = orc.moments[:, 2].sum() / n_obs
    z = (e_binned - e_exact) / (p.e_bin / math.sqrt(12.0 * n_obs))
    n_err = max(abs(Hb @ Nb - orc.moments[:, 0].sum()), abs(Hb @ Nb ** 2 - orc.moments[:, 1].sum()))
    return z, n_err


def test_binned_mean_energy_matches_exact_moments():
    z, n_err = lj_binned_mean_z()
    assert abs(z) < 5.0
    assert n_err == 0.0


def test_binned_mean_energy_catches_planted_mistakes():
    # one bin too high: +e_bin; energies taken at the lower bin edge: -e_bin / 2
    assert lj_binned_mean_z(mutation=8192)[0] > 50.0
    assert lj_binned_mean_z(centre=0.0)[0] < -25.0


def small_box_mbar_z(centre=0.5, n_runs=8, sweeps=15000, e_bin=0.05, detail=False):
    """Binned MBAR at unsampled chemical potentials of the small box against
    the brute-force <N> and <E>; returns the largest |z| over the runs' spread."""
    # E = 0 (every empty walker) at the centre of a bin, not on an edge
    base = small_box_problem().replace(e_lo=-40.0 - 0.5 * e_bin, e_bin=e_bin, n_e_bins=int(round(80.0 / e_bin)))
    bf = brute_force_small_box(base)
    kT_q = np.array([0.9, 0.9, 0.9, 1.3, 1.3, 1.3])
    mu_q = np.array([-6.0, -4.75, -3.6, -5.0, -4.4, -3.5])
    exact_n, exact_e = np.zeros(len(kT_q)), np.zeros(len(kT_q))
    for q, (kT, mu) in enumerate(zip(kT_q, mu_q)):
        z1, z2, e1, e2 = bf[float(kT)]
        zz = math.exp(mu / kT) / (base.lambda0 / math.sqrt(kT)) ** 3
        w = np.array([1.0, zz * z1, zz * zz * z2 / 2.0])
        w /= w.sum()
        exact_n[q] = w @ np.arange(3)
        exact_e[q] = w[1] * e1 + w[2] * e2
    est_n, est_e = [], []
    for r in range(n_runs):
        p = base.replace(seed=100 + r)
        orc = O.Oracle(p)
        orc.run(500, exchange_every=10, hist=False)
        orc.run(sweeps, exchange_every=10)
        assert orc.e_out.sum() == 0
        kT_s = p.kT[np.arange(p.S) // p.M]
        mu_s = p.mu[np.arange(p.S) % p.M]
        Nb, Eb, Hb = MB.occupied_bins(orc.hNE, p.e_lo, p.e_bin, centre=centre)
        f, D, _, ok = MB.solve(kT_s, mu_s, p.lambda0, orc.omega, Nb, Eb, Hb, tol=1e-11)
        assert ok
        nq, _, f_q = MB.query(kT_q, mu_q, p.lambda0, Nb, Eb, Hb, D, p.nmax)
        u = MB.reduced_potential(kT_q, mu_q, p.lambda0, Nb, Eb)
        wq = np.exp(np.log(Hb)[None, :] - u - D[None, :] + f_q[:, None])
        est_n.append(nq)
        est_e.append(wq @ Eb)
    est_n, est_e = np.array(est_n), np.array(est_e)
    zn = (est_n.mean(0) - exact_n) / np.maximum(est_n.std(0, ddof=1) / math.sqrt(n_runs), 1e-9)
    ze = (est_e.mean(0) - exact_e) / np.maximum(est_e.std(0, ddof=1) / math.sqrt(n_runs), 1e-9)
    if detail:
        return zn, ze, est_n.mean(0) - exact_n, est_e.mean(0) - exact_e, est_e.std(0, ddof=1) / math.sqrt(n_runs)
    return float(np.max(np.abs(zn))), float(np.max(np.abs(ze)))


@pytest.mark.slow
def test_small_box_binned_mbar_matches_brute_force():
    zn, ze = small_box_mbar_z()
    assert zn < 4.5 and ze < 4.5


@pytest.mark.slow
def test_small_box_binned_mbar_catches_lower_edge_energies():
    _, ze = small_box_mbar_z(centre=0.0)
    assert ze > 15.0


def cfg1_observations(sweeps=1000, burn=100):
    """Configuration 1 (16 states, Nmax 32, from N = 0), exchange every 10
    sweeps; every walker's (state, N, E) after every sweep past the burn-in,
    and the oracle holding the pooled histogram of exactly those observations."""
    p = W.fcc100_small()
    orc = O.Oracle(p)
    orc.run(burn, exchange_every=10, hist=False)
    st, nn, ee = [], [], []
    for k in range(sweeps):
        orc.sweeps(1)
        st.append(orc.state_of_walker.copy())
        nn.append(orc.n.copy())
        ee.append(orc.energy.copy())
        if (k + 1) % 10 == 0:
            orc.exchange()
    return p, orc, np.concatenate(st), np.concatenate(nn).astype(np.float64), np.concatenate(ee)


def test_cfg1_binned_against_unbinned_mbar():
    p, orc, st, N, E = cfg1_observations()
    S = p.S
    kT_s = p.kT[np.arange(S) // p.M]
    mu_s = p.mu[np.arange(S) % p.M]
    omega = np.bincount(st, minlength=S).astype(np.float64)
    # the oracle's histogram holds exactly these observations
    assert np.array_equal(orc.omega, omega.astype(np.int64))
    assert np.array_equal(orc.hN.sum(axis=0), np.bincount(N.astype(np.int64), minlength=p.nmax + 1))
    # unbinned: identical (N, E) observations (the empty walkers) pooled exactly
    key, inv, cnt = np.unique(np.stack([N, E], axis=1), axis=0, return_inverse=True, return_counts=True)
    f_u, D_u, _, ok_u = MB.solve(kT_s, mu_s, p.lambda0, omega, key[:, 0], key[:, 1], cnt.astype(float), tol=1e-9)
    kT_q = np.array([0.7, 0.9, 1.2, 1.4])
    mu_q = np.array([-5.5, -4.0, -3.0, -2.5])
    nq_u, _, _ = MB.query(kT_q, mu_q, p.lambda0, key[:, 0], key[:, 1], cnt.astype(float), D_u, p.nmax)

    def binned(hNE, centre=0.5):
        Nb, Eb, Hb = MB.occupied_bins(hNE, p.e_lo, p.e_bin, centre=centre)
        f, D, _, ok = MB.solve(kT_s, mu_s, p.lambda0, omega, Nb, Eb, Hb, tol=1e-9)
        nq, _, _ = MB.query(kT_q, mu_q, p.lambda0, Nb, Eb, Hb, D, p.nmax)
        return f, nq, ok

    f_b, nq_b, ok_b = binned(orc.hNE)
    assert ok_u and ok_b
    # binning moves each energy by at most e_bin / 2 (uniformly, mean zero): the
    # free energies move by far less than the largest systematic shift
    # max |beta_s - beta_0| e_bin / 2 that a biased bin energy would cause
    shift = np.max(np.abs(1.0 / kT_s - 1.0 / kT_s[0])) * p.e_bin / 2.0
    assert np.max(np.abs(f_b - f_u)) < 0.1 * shift
    np.testing.assert_allclose(nq_b, nq_u, rtol=2e-3, atol=2e-3)
    # bins taken at their lower edge shift f by (beta_s - beta_0) e_bin / 2
    f_edge, _, _ = binned(orc.hNE, centre=0.0)
    assert np.max(np.abs(f_edge - f_u)) > 0.8 * shift


# ---------------------------------------------- per-state energy histograms

def ideal_state_window_errors(mutation=0):
    """Ideal gas (E = 0 always) with a different window per state: the bin of
    E = 0 in each state's window is known in closed form, so every state's
    observations must sit in that one bin (underflow and overflow included)."""
    # neighbouring states close together, so that walkers often swap states
    p = W.ideal_gas(W.fcc100_small(L=2, M=3, nmax=24)).replace(kT=np.array([1.0, 1.1]),
                                                               mu=np.array([-3.0, -2.9, -2.8]))
    orc = O.Oracle(p, mutation=mutation)
    # 4 bins of 0.25 from e_lo: E = 0 lands in window bin floor(-e_lo / 0.25)
    e_lo = np.array([-0.55, 0.1, -2.0, 0.0, -1.0, -0.3])
    expect = np.array([3, 0, 5, 1, 5, 2])   # bin 2, below, beyond, bin 0, beyond (0 is the end), bin 1
    orc.set_state_windows(4, 0.25, e_lo)
    orc.run(300, exchange_every=10)
    want = np.zeros_like(orc.hE)
    want[np.arange(p.S), expect] = orc.omega
    return int(np.abs(orc.hE - want).sum()), orc


def test_ideal_gas_state_windows_exact():
    err, orc = ideal_state_window_errors()
    assert err == 0
    assert orc.ex_counts[:, :, 1].sum() > 10        # walkers did change states


def lj_state_window_z(mutation=0, n_bins=4096, e_bin=0.1):
    """Per state: z of (mean bin energy - exact mean energy) over the same
    observations, windows centred on each state's mean from an earlier run;
    +inf where an observation fell outside its window.  (The ideal gas cannot
    tell a walker's row from its state's row: every row then gets one
    observation per sweep, all at E = 0; here the energy depends on the state.)"""
    p = W.fcc100_small()
    pos, n = W.initial_walkers(p, [8] * p.S, seed=6)
    orc = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    orc.run(1500, exchange_every=10, hist=False)
    orc.run(300, exchange_every=10)
    mean = orc.moments[:, 2] / orc.omega
    orc.set_state_windows(n_bins, e_bin, mean - 0.5 * n_bins * e_bin)
    orc.reset_histograms()
    orc.run(600, exchange_every=10)
    inside = orc.hE[:, 1:-1]
    n_s = inside.sum(axis=1)
    if not np.array_equal(n_s, orc.omega):
        return np.inf
    centres = orc.hE_lo[:, None] + (np.arange(n_bins) + 0.5) * e_bin
    e_binned = (inside * centres).sum(axis=1) / n_s
    e_exact = orc.moments[:, 2] / orc.omega
    return float(np.max(np.abs(e_binned - e_exact) / (e_bin / np.sqrt(12.0 * n_s))))


def test_lj_state_windows_match_exact_moments():
    assert lj_state_window_z() < 5.0


def test_lj_state_windows_catch_walker_rows():
    assert lj_state_window_z(mutation=16384) > 20.0
