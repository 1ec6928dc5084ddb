"""FP64 oracle of the MBAR reweighting of Sec. II.B (arXiv:1908.11118).

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU baseline,
never by the library.

Samples are pooled into bins b = (N_b, E_b) with counts H_b.  State s
(kT_s, mu_s), observed Omega_s times, has the grand-canonical reduced
potential of Eq. grandpot,

    u_s(N, E) = beta_s (E - mu_s N) + 3 N ln Lambda_s,   Lambda_s = lambda0 / sqrt(kT_s).

The 3 N ln Lambda_s term is the thermal-wavelength factor of Eq. Ngrand.  It
is constant in N at fixed T, so the paper can leave it out of Eq. grandpot for
one temperature.  Across temperatures it does not cancel, and it must be kept.

Eq. normlizationconstant: c_s = sum over all samples x of
q_s(x) / sum_k Omega_k c_k^{-1} q_k(x), with q_s = exp(-u_s).  With
f_s = -ln c_s and the samples pooled by bin this is the fixed point

    D_b = ln sum_k Omega_k exp(f_k - u_k(b))
    f_s = -ln sum_b H_b exp(-u_s(b) - D_b)

gauged to f_0 = 0.  At any query state q the weight of bin b is
H_b exp(-u_q(b) - D_b + f_q), from which <N> and p_N (Eq. textbook, with the
phase indicator chi_i = [N = i]) follow.
"""
from __future__ import annotations

import numpy as np


def lse(a, axis=None):
    """log(sum(exp(a))) computed with the maximum shifted out."""
    a = np.asarray(a, np.float64)
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    out = np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True)) + m
    return np.squeeze(out, axis=axis) if axis is not None else float(out.reshape(()))


def reduced_potential(kT, mu, lambda0, N, E):
    """u(N, E) for each state (rows) and bin (columns)."""
    kT = np.atleast_1d(np.asarray(kT, np.float64))[:, None]
    mu = np.atleast_1d(np.asarray(mu, np.float64))[:, None]
    N = np.asarray(N, np.float64)[None, :]
    E = np.asarray(E, np.float64)[None, :]
    ln_lambda = np.log(lambda0) - 0.5 * np.log(kT)
    return (E - mu * N) / kT + 3.0 * N * ln_lambda


def reduced_potential2(kT, mu, mu2, lambda0, lambda0_2, N, N2, E):
    """u with a second grand-canonical species C (count N2, chemical potential
    mu2, thermal wavelength lambda0_2 / sqrt(kT)): the product over species of
    Eq. Ngrand's factors gives u = beta (E - mu N - mu2 N2) + 3 N ln Lambda
    + 3 N2 ln Lambda_C."""
    kT2 = np.atleast_1d(np.asarray(kT, np.float64))[:, None]
    mu2 = np.atleast_1d(np.asarray(mu2, np.float64))[:, None]
    N2 = np.asarray(N2, np.float64)[None, :]
    ln_lambda2 = np.log(lambda0_2) - 0.5 * np.log(kT2)
    return reduced_potential(kT, mu, lambda0, N, E) + (-mu2 / kT2 + 3.0 * ln_lambda2) * N2


def mu_from_pressure(kT, p, lambda0):
    """mu = kT ln(p Lambda^3 / kT): the ideal-gas reservoir relation of Sec. III.A
    (beta mu = beta mu0 + ln(beta p), mu0 = kT ln Lambda^3)."""
    kT = np.asarray(kT, np.float64)
    lam = lambda0 / np.sqrt(kT)
    return kT * np.log(np.asarray(p, np.float64) * lam ** 3 / kT)


def occupied_bins(hNE, e_lo, e_bin, centre: float = 0.5):
    """Pooled (N, E) histogram -> (N_b, E_b at the bin centre, H_b) of the
    non-empty bins, in row-major (N, E-bin) order.  Bin k covers
    [e_lo + k e_bin, e_lo + (k + 1) e_bin); centre is the fraction of the bin
    where its energy is taken (0.5: the midpoint; any other value is a planted
    mistake used by the tests)."""
    hNE = np.asarray(hNE)
    n_idx, k_idx = np.nonzero(hNE)
    return (n_idx.astype(np.float64), e_lo + (k_idx + centre) * e_bin,
            hNE[n_idx, k_idx].astype(np.float64))


def occupied_bins2(hNE, nmax, e_lo, e_bin):
    """Pooled (N_B, N_C, E) histogram of two species (row N_B (nmax+1) + N_C)
    -> (N_B, N_C, E at the bin centre, H) of the non-empty bins."""
    hNE = np.asarray(hNE)
    r_idx, k_idx = np.nonzero(hNE)
    return ((r_idx // (nmax + 1)).astype(np.float64), (r_idx % (nmax + 1)).astype(np.float64),
            e_lo + (k_idx + 0.5) * e_bin, hNE[r_idx, k_idx].astype(np.float64))


def solve(kT_s, mu_s, lambda0, omega_s, N_b, E_b, H_b, tol=1e-10, max_iter=200000, mu2_s=None, N2_b=None,
          lambda0_2=1.0, f0=None):
    """Self-consistent MBAR free energies f_s (f_0 = 0); with mu2_s and N2_b
    the reduced potential of two species (reduced_potential2).  The plain
    iteration starts from f0 (default 0); with max_iter=1 it applies the map
    once, so that a solution found elsewhere can be checked as a fixed point.

    Returns (f [S], D [B], iterations, converged)."""
    if N2_b is None:
        u = reduced_potential(kT_s, mu_s, lambda0, N_b, E_b)      # [S, B]
    else:
        u = reduced_potential2(kT_s, mu_s, mu2_s, lambda0, lambda0_2, N_b, N2_b, E_b)
    omega = np.asarray(omega_s, np.float64)
    ln_omega = np.where(omega > 0, np.log(np.where(omega > 0, omega, 1.0)), -np.inf)
    ln_h = np.log(np.asarray(H_b, np.float64))
    f = np.zeros(u.shape[0]) if f0 is None else np.asarray(f0, np.float64) - float(f0[0])
    it, converged = 0, False
    D = None
    while it < max_iter:
        it += 1
        D = lse(ln_omega[:, None] + f[:, None] - u, axis=0)           # [B]
        f_new = -lse(ln_h[None, :] - u - D[None, :], axis=1)          # [S]
        f_new = f_new - f_new[0]
        delta = np.max(np.abs(f_new - f))
        f = f_new
        if delta < tol:
            converged = True
            break
    D = lse(ln_omega[:, None] + f[:, None] - u, axis=0)
    return f, D, it, converged


def query(kT_q, mu_q, lambda0, N_b, E_b, H_b, D_b, nmax):
    """Reweight to query states (kT_q[i], mu_q[i]).

    Returns (<N> [Q], p_N [Q, nmax+1], f_q [Q]) where f_q is the MBAR free
    energy of the query state in the gauge of solve()."""
    u = reduced_potential(kT_q, mu_q, lambda0, N_b, E_b)          # [Q, B]
    ln_w = np.log(np.asarray(H_b, np.float64))[None, :] - u - np.asarray(D_b)[None, :]
    f_q = -lse(ln_w, axis=1)
    w = np.exp(ln_w + f_q[:, None])
    N_b = np.asarray(N_b)
    n_mean = w @ N_b
    p_N = np.zeros((u.shape[0], nmax + 1))
    for n in range(nmax + 1):
        sel = N_b == n
        if np.any(sel):
            p_N[:, n] = np.sum(w[:, sel], axis=1)
    return n_mean, p_N, f_q


def query2(kT_q, mu_q, mu2_q, lambda0, lambda0_2, N_b, N2_b, E_b, H_b, D_b, nmax):
    """Two species: reweight to query states (kT_q, mu_q, mu2_q).

    Returns (<N_B> [Q], <N_C> [Q], p_N_B [Q, nmax+1], p_N_C [Q, nmax+1], f_q [Q])."""
    u = reduced_potential2(kT_q, mu_q, mu2_q, lambda0, lambda0_2, N_b, N2_b, E_b)
    ln_w = np.log(np.asarray(H_b, np.float64))[None, :] - u - np.asarray(D_b)[None, :]
    f_q = -lse(ln_w, axis=1)
    w = np.exp(ln_w + f_q[:, None])
    N_b, N2_b = np.asarray(N_b), np.asarray(N2_b)
    pB = np.zeros((u.shape[0], nmax + 1))
    pC = np.zeros((u.shape[0], nmax + 1))
    for n in range(nmax + 1):
        pB[:, n] = np.sum(w[:, N_b == n], axis=1)
        pC[:, n] = np.sum(w[:, N2_b == n], axis=1)
    return w @ N_b, w @ N2_b, pB, pC, f_q
