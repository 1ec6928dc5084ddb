"""GPU parity of the cluster-in-gas system (a second mobile species that only
displaces; insertion and removal on the grand-canonical species).

* Lock-step traces against the FP64 oracle, plain and delayed acceptance, on a
  16-replica cluster-in-gas system, then final states, histograms (over N_B)
  and counters; exact running energies.
* The 4096-replica, Nmax_B 64 workload in the launch configuration the
  benchmark times: two traced sweeps against the oracle.
* Walkers without the cluster are refused, and so is sweeping before walkers
  are supplied; a batch with cluster members equals stepping them one by one.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Batch, Regc
from paper_1908_11118_gb300 import build as B
from test_gpu_parity import assert_same_state, run_lockstep
from test_gpu_surrogate import assert_same_final_state, run_da_lockstep, theta_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def small_cluster_problem(seed=0):
    return W.cluster_in_gas(L=4, M=4, nmax_b=64, seed=seed)


def test_lockstep_cluster_16_replicas():
    p = small_cluster_problem()
    rng = np.random.default_rng(0)
    pos, n = W.cluster_initial(p, rng.integers(0, 40, p.S), seed=1)
    g, o, compared, diverged, observed = run_lockstep(p, pos, n, blocks=8, sweeps=10, min_moves=p.S * 20 * 10)
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0
    # the cluster atoms are still particles 0..3 of every walker
    pg, ng, _, _ = g.get_walkers()
    assert np.all(ng >= p.n_cluster)


def test_lockstep_cluster_delayed_acceptance():
    p = small_cluster_problem(seed=2)
    rng = np.random.default_rng(1)
    pos, n = W.cluster_initial(p, rng.integers(0, 30, p.S), seed=3)
    g, o, compared, exact, diverged, screened, passed = run_da_lockstep(p, pos, n, theta_of(2), blocks=6,
                                                                        sweeps=10)
    assert 0 < passed < screened
    if not diverged:
        assert_same_final_state(g, o, p, screened, passed)


def test_full_size_cluster_4096_replicas():
    p = W.cluster_in_gas()
    rng = np.random.default_rng(0)
    pos, n = W.cluster_initial(p, rng.integers(0, 33, p.S), seed=0)
    g, o, compared, diverged, observed = run_lockstep(p, pos, n, blocks=1, sweeps=2, exchange=True,
                                                      min_moves=p.S * 40 // 2)
    assert len(diverged) <= 2
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0


def test_cluster_walker_checks():
    p = small_cluster_problem()
    g = Regc(p)
    with pytest.raises(Exception):
        g.sweep(1)                          # no walkers with the cluster yet
    pos, n = W.cluster_initial(p, 5, seed=4)
    bad = n.copy()
    bad[3] = p.n_cluster - 1
    with pytest.raises(Exception):
        g.set_walkers(pos, bad)
    g.set_walkers(pos, n)
    g.sweep(2)
    assert np.all(g.get_walkers()[1] >= p.n_cluster)
    h = g.histograms()["hN"]
    assert h[:, p.nmax - p.n_cluster + 1:].sum() == 0     # histograms over N_B


def test_batch_with_cluster_members():
    ps = [small_cluster_problem(seed=s) for s in (5, 6)] + [W.fcc100_small(L=2, M=2, seed=7)]
    def make():
        hs = []
        for i, p in enumerate(ps):
            if p.n_cluster:
                pos, n = W.cluster_initial(p, 10 + i, seed=i)
            else:
                pos, n = W.initial_walkers(p, 6, seed=i)
            h = Regc(p)
            h.set_walkers(pos, n)
            hs.append(h)
        return hs
    A, Bs = make(), make()
    with Batch(A, sweeps_per_step=5) as bt:
        bt.run(3)
        bt.sync()
    for h in Bs:
        for _ in range(3):
            h.sweep(5)
            h.exchange()
    for a, b in zip(A, Bs):
        for x, y in zip(a.get_walkers(), b.get_walkers()):
            assert np.array_equal(x, y)
        assert np.array_equal(a.histograms()["hN"], b.histograms()["hN"])


def test_lockstep_cluster_on_a_slab():
    """A cluster species of its own potential type (2) above the fcc(100)
    slab: cluster-surface pairs use eps/sigma[2][1], cluster-gas [0][2],
    cluster-cluster [2][2]."""
    base = W.fcc100_small(L=2, M=2, nmax=40, seed=8)
    eps, sig = base.eps.copy(), base.sigma.copy()
    eps[2, 2], sig[2, 2] = 1.5, 1.05
    eps[0, 2] = eps[2, 0] = 1.2
    eps[1, 2] = eps[2, 1] = 1.8
    p = base.replace(n_types=3, eps=eps, sigma=sig, n_cluster=3, cluster_type=2)
    # cluster atoms close to the surface (within rc of the top layer), then gas
    rng = np.random.default_rng(4)
    pos = np.zeros((p.S, p.nmax, 3))
    n = np.zeros(p.S, np.int32)
    for w in range(p.S):
        clus = np.array([[1.0, 1.0, p.z_lo + 1.0], [2.2, 1.0, p.z_lo + 1.1], [1.6, 2.1, p.z_lo + 1.0]])
        pos[w, :3] = W.f32(clus)
        k = 0
        while k < 8 + 2 * w:
            q = W.f32(rng.uniform([0, 0, p.z_lo + 0.5], [p.Lx, p.Ly, p.z_hi]))
            d = q - pos[w, :3 + k]
            d[:, :2] -= np.round(d[:, :2] / [p.Lx, p.Ly]) * [p.Lx, p.Ly]
            if np.min(np.linalg.norm(d, axis=1)) > 0.95:
                pos[w, 3 + k] = q
                k += 1
        n[w] = 3 + k
    g, o, compared, diverged, observed = run_lockstep(p, pos, n, blocks=6, sweeps=10, min_moves=p.S * 20 * 6)
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0
