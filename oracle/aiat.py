"""FP64 oracle of aiAT@REGC (Sec. III.A.1, Eq. aiTherm).

TEST INFRASTRUCTURE ONLY: used by the tests, never by the library.

For every composition N_B seen among the samples, the sample of lowest
energy is selected; with the free energies approximated by those energies
(all vibrational contributions assumed to cancel) the formation free energy
of composition n at chemical potential mu is

    dG(n; mu) = E_min(n) - E_min(0) - n mu,

E_min(0) being the energy of the pristine slab (0 with the frozen slab's own
interactions left out, as in the energies here).  At each state the stable
composition is the n of lowest dG (ties: the smaller n).  The temperature
enters only through mu(T, p).
"""
from __future__ import annotations

import numpy as np


def lowest_energy(N, E, nmax):
    """E_min [nmax + 1] (NaN where no sample has that N) and the index of the
    first sample attaining it (-1 where none)."""
    N = np.asarray(N)
    E = np.asarray(E, np.float64)
    e_min = np.full(nmax + 1, np.nan)
    first = np.full(nmax + 1, -1, np.int64)
    for i in range(len(N)):
        n = int(N[i])
        if first[n] < 0 or E[i] < e_min[n]:
            e_min[n] = E[i]
            first[n] = i
    return e_min, first


def formation_free_energy(e_min, mu_q, e_pristine=0.0):
    """dG [Q, nmax + 1] (+inf where the composition was not seen) and the
    stable composition [Q] at each chemical potential."""
    mu_q = np.atleast_1d(np.asarray(mu_q, np.float64))
    n = np.arange(len(e_min))
    seen = ~np.isnan(e_min)
    dG = np.where(seen[None, :], np.nan_to_num(e_min)[None, :] - e_pristine - n[None, :] * mu_q[:, None], np.inf)
    return dG, np.argmin(dG, axis=1)
