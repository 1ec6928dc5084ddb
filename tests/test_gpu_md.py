"""GPU tests of the REGCMD segment (regc_md) against the FP64 oracle.

MD trajectories from binary32 and FP64 arithmetic separate over time, so the
parity of a segment is a short one: from identical walkers and Philox
streams, five steps of the GPU and the oracle end within a position
tolerance, with matching kinetic and potential energies.  The sampling itself
is checked statistically against values the oracle's pins fix:
  * MD alone gives one particle above the small box's surface its
    brute-force canonical mean energy at every temperature;
  * the thermostat keeps the kinetic energy of an ideal gas at its canonical
    mean and variance;
  * grand-canonical sweeps alternated with MD segments reproduce the
    brute-force <N> and <E> of the small box;
and for the cluster species a short segment matches the oracle too.  The
REGCMD cycle (the x0 choice of Sec. II.A, then an MD segment) makes the same
exchanges as the oracle's over a few steps and reproduces the small box's
brute-force averages.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Regc
from paper_1908_11118_gb300 import build as B
from test_md_oracle import expected_small_box
from test_oracle_pins import brute_force_small_box, small_box_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def short_segment_parity(p, pos, n, steps=5, dt=0.002, tau=0.05):
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    kg = g.md(steps, dt, tau)
    ko = o.md(steps, dt, tau)
    pg, ng, eg, _ = g.get_walkers()
    L = np.array([p.Lx, p.Ly, p.Lz])
    worst = 0.0
    for w in range(p.S):
        if n[w] == 0:
            continue
        d = pg[w, :n[w]] - o.pos[w, :n[w]]
        d[:, :2] -= np.round(d[:, :2] / L[:2]) * L[:2]
        if p.periodic_z:
            d[:, 2] -= np.round(d[:, 2] / L[2]) * L[2]
        worst = max(worst, float(np.max(np.abs(d))))
    print("worst position difference after %d steps: %.3g" % (steps, worst))
    assert worst < 2e-5, worst
    np.testing.assert_allclose(kg, ko, rtol=2e-4, atol=1e-4)
    np.testing.assert_allclose(eg, o.energy, rtol=1e-4, atol=2e-3)
    assert g.check_energy() == 0.0
    return g, o


def test_short_segment_matches_oracle_slab():
    p = W.fcc100_small(seed=1)
    rng = np.random.default_rng(3)
    pos, n = W.initial_walkers(p, rng.integers(0, 25, p.S), seed=2)
    short_segment_parity(p, pos, n)


def test_short_segment_matches_oracle_cluster():
    p = W.cluster_in_gas(L=2, M=2, nmax_b=40, seed=2)
    pos, n = W.cluster_initial(p, [0, 10, 25, 40], seed=5)
    short_segment_parity(p, pos, n)


def test_md_alone_gives_the_canonical_energy_of_one_particle():
    p = small_box_problem()
    pos = np.zeros((p.S, p.nmax, 3))
    pos[:, 0] = [1.3, 1.3, 2.0]
    g = Regc(p)
    g.set_walkers(pos, np.ones(p.S, np.int32))
    es = []
    for k in range(3000):
        g.md(25, 0.005, 0.05, kinetic=False)
        es.append(g.get_walkers()[2])
    es = np.array(es)[300:]
    b = es[: len(es) // 20 * 20].reshape(20, -1, p.S).mean(axis=1)
    bf = brute_force_small_box(p)
    for s in range(p.S):
        e1 = bf[float(p.kT[s // p.M])][2]
        z = (b[:, s].mean() - e1) / (b[:, s].std(ddof=1) / math.sqrt(20))
        assert abs(z) < 4.5, (s, b[:, s].mean(), e1, z)


def test_thermostat_canonical_kinetic_energy():
    p = W.ideal_gas(W.fcc100_small(L=1, M=2, seed=4))
    pos, n = W.initial_walkers(p, 10, seed=6)
    g = Regc(p)
    g.set_walkers(pos, n)
    ks = np.array([g.md(40, 0.01, 0.05) for _ in range(400)])
    sow = g.get_walkers()[3]
    for w in range(p.S):
        kT = p.kT[sow[w] // p.M]
        nf = 3 * int(n[w])
        mean, var = nf * kT / 2, nf * kT * kT / 2
        z_mean = (ks[:, w].mean() - mean) / math.sqrt(var / len(ks))
        a = nf / 2
        z_var = (ks[:, w].var(ddof=1) - var) / math.sqrt(kT ** 4 * (2 * a * a + 6 * a) / len(ks))
        assert abs(z_mean) < 4.5 and abs(z_var) < 4.5, (w, z_mean, z_var)


def test_regcmd_small_box_brute_force():
    p = small_box_problem().replace(p_disp=0.0, moves_per_sweep=4)
    g = Regc(p)
    nb, eb = [], []
    nv = np.arange(p.nmax + 1)
    prev = g.histograms()
    for b in range(16):
        for c in range(375):
            g.sweep(1)
            g.md(10, 0.005, 0.1, kinetic=False)
            if c % 10 == 9:
                g.exchange()
        h = g.histograms()
        dh = h["hN"] - prev["hN"]
        nb.append((dh @ nv) / np.maximum(dh.sum(axis=1), 1))
        eb.append((h["moments"][:, 2] - prev["moments"][:, 2]) / np.maximum(h["omega"] - prev["omega"], 1))
        prev = h
    nb, eb = np.array(nb), np.array(eb)
    exp_n, exp_e, _ = expected_small_box(p)
    zn = (nb.mean(axis=0) - exp_n) / (nb.std(axis=0, ddof=1) / 4.0)
    ze = (eb.mean(axis=0) - exp_e) / (eb.std(axis=0, ddof=1) / 4.0)
    assert max(np.max(np.abs(zn)), np.max(np.abs(ze))) < 4.5, (zn, ze)


def test_md_arguments_and_checkpoint():
    p = W.fcc100_small(L=1, M=2, seed=7)
    pos, n = W.initial_walkers(p, 8, seed=1)
    g = Regc(p)
    g.set_walkers(pos, n)
    for bad in ((-1, 0.01, 0.1), (5, 0.0, 0.1), (5, 0.01, 0.0)):
        with pytest.raises(Exception):
            g.md(*bad)
    g.md(5, 0.002, 0.05)
    ck = g.checkpoint()
    g.md(5, 0.002, 0.05)
    want = g.get_walkers()
    h = Regc(p)
    h.restore(ck)
    h.md(5, 0.002, 0.05)
    for x, y in zip(h.get_walkers(), want):
        assert np.array_equal(x, y)      # the MD streams continue exactly


def test_regcmd_cycle_short_parity():
    """A few REGCMD steps (the x0 choice, then five MD steps) from identical
    walkers: the same particle and replica exchanges as the oracle, positions
    within the MD tolerance."""
    p = W.fcc100_small(seed=5)
    rng = np.random.default_rng(8)
    pos, n = W.initial_walkers(p, rng.integers(2, 20, p.S), seed=4)
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    for _ in range(3):
        assert g.cycle_md(2, 0.7, 5, 0.002, 0.05) == o.cycle_md(2, 0.7, 5, 0.002, 0.05)
    pg, ng, eg, sg = g.get_walkers()
    assert np.array_equal(ng, o.n) and np.array_equal(sg, o.state_of_walker)
    L = np.array([p.Lx, p.Ly])
    for w in range(p.S):
        d = pg[w, :ng[w]] - o.pos[w, :ng[w]]
        d[:, :2] -= np.round(d[:, :2] / L) * L
        assert np.max(np.abs(d), initial=0.0) < 1e-4, w
    np.testing.assert_allclose(eg, o.energy, rtol=1e-4, atol=2e-3)
    mv, ex, _ = g.counters()
    assert np.array_equal(mv, o.counts) and np.array_equal(ex, o.ex_counts)
    assert mv[:, 0, 0].sum() == 0                          # no displacement moves: MD does the diffusion


def test_regcmd_cycle_small_box_brute_force():
    p = small_box_problem().replace(p_disp=0.0)
    g = Regc(p)
    nb, eb = [], []
    nv = np.arange(p.nmax + 1)
    prev = g.histograms()
    for b in range(16):
        g.cycle_md(375, 0.9, 10, 0.005, 0.1)
        h = g.histograms()
        dh = h["hN"] - prev["hN"]
        nb.append((dh @ nv) / np.maximum(dh.sum(axis=1), 1))
        eb.append((h["moments"][:, 2] - prev["moments"][:, 2]) / np.maximum(h["omega"] - prev["omega"], 1))
        prev = h
    nb, eb = np.array(nb), np.array(eb)
    exp_n, exp_e, _ = expected_small_box(p)
    zn = (nb.mean(axis=0) - exp_n) / (nb.std(axis=0, ddof=1) / 4.0)
    ze = (eb.mean(axis=0) - exp_e) / (eb.std(axis=0, ddof=1) / 4.0)
    assert max(np.max(np.abs(zn)), np.max(np.abs(ze))) < 4.5, (zn, ze)
    for bad in ((5, 1.5, 10, 0.005, 0.1), (5, 0.5, -1, 0.005, 0.1), (5, 0.5, 10, 0.0, 0.1)):
        with pytest.raises(Exception):
            g.cycle_md(*bad)
