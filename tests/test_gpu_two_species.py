"""GPU parity of two grand-canonical species on a (T, mu_B, mu_C) grid
(regc_init_grid2: more than one reactive gas, the outlook of Sec. IV)
against the FP64 oracle.

* Lock-step: every move of every walker (species picked, particle, energy
  change, decision) over sweeps and replica exchanges along all five
  directions, then positions bit for bit, N and N_B per walker, state labels,
  the N_B and N_C histograms, the moments and the counters; the running
  energy equals the from-scratch one exactly.
* The ideal gas with exchange: per-state <N_B>, <N_C> against the product of
  two Poisson laws truncated to N_B + N_C <= Nmax, within 3 standard errors.
* Walker upload with species counts, energies against the oracle's.
* Checkpoint and resume; the paths that take one species only refuse.
* MBAR over the (N_B, N_C, E) histogram (regc_reweight2): the sampled
  states' free energies and the reweighted means and distributions of both
  counts against oracle/mbar.py on the same bins.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mbar as OM
from oracle import oracle as O
from paper_1908_11118_gb300 import Batch, Regc
from paper_1908_11118_gb300 import build as B
from parity import compare_traces
from test_two_species_oracle import trunc_joint_means

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def make(p, nb, nc, seed):
    pos, n, nbv = W.two_gas_initial(p, nb, nc, seed=seed)
    g = Regc(p)
    g.set_walkers(pos, n, nb=nbv)
    o = O.Oracle(p, pos=pos, n=n, nb=nbv)
    return g, o


def test_energies_of_uploaded_walkers():
    p = W.two_gas_small()
    rng = np.random.default_rng(2)
    g, o = make(p, rng.integers(0, 15, p.S), rng.integers(0, 15, p.S), seed=4)
    _, n, e, _ = g.get_walkers()
    assert np.array_equal(n, o.n) and np.array_equal(g.species_counts(), o.nb)
    assert np.all(np.abs(e - o.energy) <= 1e-5 * np.maximum(1.0, np.abs(o.energy)))
    assert g.check_energy() == 0.0


def test_lockstep_two_species():
    p = W.two_gas_small()
    rng = np.random.default_rng(7)
    g, o = make(p, rng.integers(0, 12, p.S), rng.integers(0, 12, p.S), seed=5)
    beta_max = 1.0 / float(np.min(p.kT))
    compared = 0
    diverged = []
    for block in range(8):
        tg = g.sweep_traced(10)
        to = o.sweeps(10, trace=True)
        c, d = compare_traces(tg, to, beta_max)
        compared += c
        if d:
            diverged = d
            break
        g.exchange()
        o.exchange()
    assert compared >= p.S * 20 * 10
    gm = (tg["type"] > 0).sum()
    assert gm > 0
    if diverged:
        pytest.skip("the chains parted at a near tie (checked by compare_traces)")
    pos, n, e, sow = g.get_walkers()
    assert np.array_equal(n, o.n)
    assert np.array_equal(g.species_counts(), o.nb)
    assert np.array_equal(sow, o.state_of_walker)
    for w in range(p.S):
        assert np.array_equal(pos[w, :n[w]], o.pos[w, :n[w]].astype(np.float32)), w
    assert np.all(np.abs(e - o.energy) <= 1e-4 * np.maximum(1.0, np.abs(o.energy)))
    h = g.histograms()
    assert np.array_equal(h["hN"], o.hN) and np.array_equal(h["hN2"], o.hN2)
    assert np.array_equal(h["omega"], o.omega)
    np.testing.assert_allclose(h["moments"][:, :2], o.moments[:, :2], rtol=1e-12)
    np.testing.assert_allclose(h["moments2"], o.moments2, rtol=1e-12)
    assert int(h["hNE"].sum()) + int(h["e_out"].sum()) == int(o.hNE.sum()) + int(o.e_out.sum())
    mv, ex, _ = g.counters()
    assert np.array_equal(mv, o.counts) and np.array_equal(ex, o.ex_counts)
    assert ex[:, 4, 0].sum() > 0                      # the mu_C direction was drawn
    assert (o.nb > 0).any() and (o.n - o.nb > 0).any()
    assert g.check_energy() == 0.0


def test_ideal_gas_two_species_on_gpu():
    p = W.ideal_gas(W.two_gas_small(L=2, M=3, K=3, nmax=16)).replace(
        kT=np.array([0.9, 1.1]), mu=np.array([-4.6, -4.3, -4.0]), mu2=np.array([-4.8, -4.4, -4.0]),
        moves_per_sweep=4, p_disp=0.0)
    g = Regc(p)
    kT, mu, mu2 = p.state_params()
    exp_b, exp_c = np.zeros(p.S), np.zeros(p.S)
    for s in range(p.S):
        lb = p.volume * math.exp(mu[s] / kT[s]) / (p.lambda0 / math.sqrt(kT[s])) ** 3
        lc = p.volume * math.exp(mu2[s] / kT[s]) / (p.lambda0_2 / math.sqrt(kT[s])) ** 3
        exp_b[s], exp_c[s], _ = trunc_joint_means(lb, lc, p.nmax)
    g.run(200, exchange_every=1)
    nb_m, nc_m = [], []
    nv = np.arange(p.nmax + 1)
    prev = g.histograms()
    for b in range(40):
        g.run(500, exchange_every=1)
        h = g.histograms()
        d, d2 = h["hN"] - prev["hN"], h["hN2"] - prev["hN2"]
        nb_m.append((d @ nv) / np.maximum(d.sum(1), 1))
        nc_m.append((d2 @ nv) / np.maximum(d2.sum(1), 1))
        prev = h
    for m, ex in ((np.array(nb_m), exp_b), (np.array(nc_m), exp_c)):
        se = np.maximum(m.std(0, ddof=1) / math.sqrt(len(m)), 1e-3)
        z = np.abs(m.mean(0) - ex) / se
        assert z.max() < 3.0, (z, m.mean(0), ex)


def test_checkpoint_and_refusals_two_species():
    p = W.two_gas_small(seed=3)
    g, _ = make(p, 6, 4, seed=1)
    g.run(30)
    ck = g.checkpoint()
    g.run(30)
    want = (g.get_walkers(), g.species_counts(), g.histograms())
    h, _ = make(p, 1, 1, seed=2)
    h.restore(ck)
    h.run(30)
    for x, y in zip(h.get_walkers(), want[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(h.species_counts(), want[1])
    for k in ("hN", "hN2", "hNE", "moments2"):
        assert np.array_equal(h.histograms()[k], want[2][k])
    single = Regc(W.fcc100_small(L=2, M=3))
    with pytest.raises(Exception):
        single.restore(ck)
    for call in (lambda: g.md(5, 0.005, 0.1), lambda: g.cycle(5, 0.9, 5), lambda: g.set_mode(True),
                 lambda: g.reweight([1.0], [-3.0]), lambda: Batch([g], 5),
                 lambda: g.structure_init(10, 0.1, [], 5, 0.1, 100)):
        with pytest.raises(Exception):
            call()


def test_reweight2_matches_oracle():
    p = W.two_gas_small(seed=11)
    g, _ = make(p, 6, 6, seed=3)
    g.run(400, exchange_every=1)
    h = g.histograms()
    assert (h["omega"] > 0).all()
    kT_s, mu_s, mu2_s = p.state_params()
    N_b, N2_b, E_b, H_b = OM.occupied_bins2(h["hNE"], p.nmax, p.e_lo, p.e_bin)
    assert len(np.unique(N2_b)) > 3 and len(np.unique(N_b)) > 3
    f_o, D_o, _, ok = OM.solve(kT_s, mu_s, p.lambda0, h["omega"].astype(float), N_b, E_b, H_b, tol=1e-12,
                               mu2_s=mu2_s, N2_b=N2_b, lambda0_2=p.lambda0_2)
    assert ok
    # queries: two sampled states and points between and beyond the grid
    kq = np.array([kT_s[0], kT_s[-1], 0.5 * (p.kT[0] + p.kT[-1]), p.kT[0]])
    mq = np.array([mu_s[0], mu_s[-1], 0.5 * (p.mu[0] + p.mu[-1]), p.mu[-1] + 0.1])
    m2q = np.array([mu2_s[0], mu2_s[-1], 0.5 * (p.mu2[0] + p.mu2[-1]), p.mu2[0] - 0.1])
    nb_o, nc_o, pb_o, pc_o, _ = OM.query2(kq, mq, m2q, p.lambda0, p.lambda0_2, N_b, N2_b, E_b, H_b, D_o, p.nmax)
    nb_g, nc_g, pb_g, pc_g, f_g, it = g.reweight2(kq, mq, m2q, tol=1e-11)
    assert it > 0
    np.testing.assert_allclose(f_g, f_o, atol=1e-8)
    np.testing.assert_allclose(nb_g, nb_o, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(nc_g, nc_o, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(pb_g, pb_o, atol=1e-9)
    np.testing.assert_allclose(pc_g, pc_o, atol=1e-9)
    np.testing.assert_allclose(pb_g.sum(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(pc_g.sum(1), 1.0, atol=1e-12)
    single = Regc(W.fcc100_small(L=2, M=3))
    single.run(20)
    with pytest.raises(Exception):
        single.reweight2([1.0], [-3.0], [-3.0])
