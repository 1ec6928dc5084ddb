"""Pins of the aiAT@REGC oracle (Sec. III.A.1, Eq. aiTherm).

* Energies linear in n, E_min(n) = -eps n: the stable composition jumps from
  the pristine slab to the largest n exactly at mu = -eps.
* Convex energies E_min(n) = a n^2 - b n: the stable composition at mu is the
  integer nearest to (b + mu) / (2 a), clipped to the seen range.
* Unseen compositions never win; the lowest energy per composition is the
  minimum over the samples, the first sample attaining it on ties.
* A sample set drawn by the oracle's REGC run: every composition's E_min is
  attained by one of the samples, and no sample of that composition lies
  below it.
"""
import numpy as np

import workloads as W
from oracle import aiat as AI
from oracle import oracle as O


def test_linear_energies_switch_at_minus_eps():
    eps, nmax = 1.7, 12
    e_min = -eps * np.arange(nmax + 1)
    _, ph = AI.formation_free_energy(e_min, [-eps - 1e-9, -eps + 1e-9, -3.0, 0.0])
    assert list(ph) == [0, nmax, 0, nmax]


def test_convex_energies_follow_the_closed_form():
    a, b, nmax = 0.25, 3.0, 20
    n = np.arange(nmax + 1)
    e_min = a * n * n - b * n
    for mu in np.linspace(-4.0, 6.0, 101):
        _, ph = AI.formation_free_energy(e_min, [mu])
        want = int(np.clip(np.floor((b + mu) / (2 * a) + 0.5), 0, nmax))
        x = (b + mu) / (2 * a)
        if abs(x - np.floor(x) - 0.5) > 1e-9:          # away from exact ties
            assert ph[0] == want, (mu, ph[0], want)


def test_unseen_compositions_and_ties():
    N = np.array([0, 2, 2, 5, 5, 5])
    E = np.array([0.0, -3.0, -4.0, -9.0, -11.0, -11.0])
    e_min, first = AI.lowest_energy(N, E, 6)
    assert np.isnan(e_min[1]) and first[1] == -1
    assert e_min[2] == -4.0 and first[2] == 2
    assert e_min[5] == -11.0 and first[5] == 4              # the first of the tied samples
    dG, ph = AI.formation_free_energy(e_min, [-2.5, -1.0])
    assert np.isinf(dG[0, 1]) and np.isinf(dG[0, 6])
    # mu = -2.5: dG = 0, 1, 1.5 for n = 0, 2, 5; mu = -1: 0, -2, -6
    assert list(ph) == [0, 5]


def test_lowest_energy_over_an_oracle_run():
    p = W.fcc100_small(seed=3)
    o = O.Oracle(p)
    Ns, Es = [], []
    for b in range(40):
        o.run(5, exchange_every=5, hist=False)
        Ns.append(o.n.copy())
        Es.append(o.energy.copy())
    N, E = np.concatenate(Ns), np.concatenate(Es)
    e_min, first = AI.lowest_energy(N, E, p.nmax)
    for n in range(p.nmax + 1):
        sel = N == n
        if not sel.any():
            assert first[n] == -1
            continue
        assert N[first[n]] == n and E[first[n]] == e_min[n]
        assert np.all(E[sel] >= e_min[n])
