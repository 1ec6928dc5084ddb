"""GPU parity of the REGC cycle (regc_cycle: Sec. II.A, Fig. 1; Sec. III.A's
x0 = 0.99 and ten MC moves per step) against the FP64 oracle.

* Lock-step traces, move by move, on the 16-replica fcc(100) system at the
  paper's x0 = 0.99 and at x0 = 0.5 (a replica exchange every other step, so
  that many launches start with a skipped particle exchange), then the final
  walkers, histograms and move and exchange counters.
* The paper's LJ surface system in eV and Angstrom (two A18 cells, 160
  replicas) in the launch configuration the benchmark times.
* Delayed acceptance and the cluster species under the cycle.
* Cycles mixed with sweeps continue one step counter; x0 = 1 and x0 = 0;
  argument checks; a checkpoint taken between cycles resumes exactly.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Regc
from paper_1908_11118_gb300 import build as B
from parity import compare_da_traces, compare_traces
from test_gpu_parity import assert_same_state, beta_max
from test_gpu_surrogate import assert_same_final_state, sur_tol_of, theta_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def run_cycle_lockstep(p, pos, n, blocks, steps, x0, n_c, min_moves=1):
    """GPU and oracle cycles side by side, compared block by block.  Returns
    (gpu, oracle, compared, diverged, observed, exchange steps)."""
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    compared, diverged, observed, n_ex = 0, [], [], 0
    for b in range(blocks):
        e0 = o.energy.copy()
        tg, xg = g.cycle_traced(steps, x0, n_c)
        to, xo = o.cycle(steps, x0, n_c, trace=True)
        assert xg == xo
        n_ex += xo
        assert np.array_equal(tg["type"] == -1, to["type"] == -1)
        de = np.where(to["accepted"] == 1, to["dE"], 0.0).sum(axis=2)
        observed.append(e0[:, None] + np.cumsum(de, axis=1))
        c, d = compare_traces(tg, to, beta_max(p))
        compared += c
        if d:
            diverged = d
            break
    assert compared >= min_moves
    return g, o, compared, diverged, np.concatenate(observed, axis=1).ravel(), n_ex


@pytest.mark.parametrize("x0", [0.99, 0.5])
def test_lockstep_fcc100_16_replicas(x0):
    p = W.fcc100_small(seed=4)
    rng = np.random.default_rng(2)
    pos, n = W.initial_walkers(p, rng.integers(0, 25, p.S), seed=3)
    g, o, compared, diverged, observed, n_ex = run_cycle_lockstep(p, pos, n, blocks=6, steps=40, x0=x0, n_c=10,
                                                                  min_moves=p.S * 10 * 40 * 3)
    assert n_ex > 0
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0


def test_lockstep_without_canonical_moves():
    """n_canonical = 0 (the REGCMD step): only the particle exchanges, each
    observed; replica-exchange steps make no move and no observation."""
    p = W.fcc100_small(seed=14)
    pos, n = W.initial_walkers(p, 9, seed=5)
    g, o, compared, diverged, observed, n_ex = run_cycle_lockstep(p, pos, n, blocks=4, steps=60, x0=0.7, n_c=0)
    assert n_ex > 0
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.histograms()["omega"].sum() == p.S * (4 * 60 - n_ex)


def test_paper_lj_slab_160_replicas():
    """The LJ A18 system (two cells) at the benchmark's settings: x0 = 0.99,
    ten displacements per step, walkers from empty to a full first layer of
    hollow sites with more B above."""
    p = W.lj_a18_slab(nmax=96, seed=1)
    rng = np.random.default_rng(5)
    pos, n = W.lj_a18_initial(p, rng.integers(0, 80, p.S), seed=6)
    g, o, compared, diverged, observed, n_ex = run_cycle_lockstep(p, pos, n, blocks=2, steps=150, x0=0.99, n_c=10,
                                                                  min_moves=p.S * 10 * 150)
    assert len(diverged) <= 2
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0


def test_delayed_acceptance_under_the_cycle():
    p = W.fcc100_small(seed=6)
    pos, n = W.initial_walkers(p, 14, seed=2)
    th = theta_of(3)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.surrogate_set(th)
    g.set_mode(True)
    o = O.Oracle(p, pos=pos, n=n, surrogate=th)
    beta = np.full(p.S, beta_max(p))
    compared = screened = passed = 0
    for b in range(4):
        tg, xg = g.cycle_traced(30, 0.9, 10)
        to, xo = o.cycle(30, 0.9, 10, trace=True)
        assert xg == xo
        c, x, d = compare_da_traces(tg, to, beta, sur_tol_of)
        compared += c
        ev = to["status"] == 0
        screened += int(ev.sum())
        passed += int((to["stage1"][ev] == 1).sum())
        if d:
            return
    assert 0 < passed < screened
    assert_same_final_state(g, o, p, screened, passed)


def test_cluster_under_the_cycle():
    p = W.cluster_in_gas(L=4, M=4, nmax_b=64, seed=3)
    rng = np.random.default_rng(3)
    pos, n = W.cluster_initial(p, rng.integers(0, 40, p.S), seed=2)
    g, o, compared, diverged, observed, n_ex = run_cycle_lockstep(p, pos, n, blocks=4, steps=40, x0=0.9, n_c=10)
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert np.all(g.get_walkers()[1] >= p.n_cluster)


def test_cycles_and_sweeps_share_the_step_counter():
    p = W.fcc100_small(L=2, M=2, seed=8)
    pos, n = W.initial_walkers(p, 8, seed=1)
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    g.sweep(3)
    o.sweeps(3)
    assert g.cycle(25, 0.8, 4) == o.cycle(25, 0.8, 4)[1]
    g.exchange()
    o.exchange()
    g.sweep(2)
    o.sweeps(2)
    assert g.cycle(25, 0.8, 4) == o.cycle(25, 0.8, 4)[1]
    pg, ng, eg, sg = g.get_walkers()
    assert np.array_equal(ng, o.n) and np.array_equal(sg, o.state_of_walker)
    for w in range(p.S):
        assert np.array_equal(pg[w, :ng[w]], o.pos[w, :ng[w]].astype(np.float32))
    mv, ex, _ = g.counters()
    assert np.array_equal(mv, o.counts) and np.array_equal(ex, o.ex_counts)


def test_x0_limits_and_arguments():
    p = W.fcc100_small(L=2, M=2, seed=9)
    pos, n = W.initial_walkers(p, 6, seed=2)
    g = Regc(p)
    g.set_walkers(pos, n)
    assert g.cycle(20, 1.0, 3) == 0
    assert g.cycle(20, 0.0, 3) == 20
    mv, ex, _ = g.counters()
    assert mv[:, 1:, 0].sum() == 20 * p.S                # one GC trial per walker and x0 = 1 step
    assert mv[:, 0, 0].sum() == 40 * 3 * p.S
    for bad in ((-1, 0.5, 3), (5, 1.5, 3), (5, -0.1, 3), (5, float("nan"), 3), (5, 0.5, -1), (5, 0.5, 1024)):
        with pytest.raises(Exception):
            g.cycle(*bad)
    assert g.cycle(0, 0.5, 3) == 0


def test_checkpoint_between_cycles():
    p = W.fcc100_small(seed=10)
    pos, n = W.initial_walkers(p, 10, seed=4)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.cycle(30, 0.9, 10)
    ck = g.checkpoint()
    g.cycle(60, 0.9, 10)
    want = g.get_walkers()
    h = Regc(p)
    h.restore(ck)
    h.cycle(60, 0.9, 10)
    for x, y in zip(h.get_walkers(), want):
        assert np.array_equal(x, y)


def test_longest_step_and_single_replica():
    """n_canonical = 1023 (the longest step a launch takes) and a grid of one
    state, where a replica-exchange attempt has no pair: the same moves as
    the oracle."""
    base = W.fcc100_small(L=1, M=1, nmax=32, seed=16)
    pos, n = W.initial_walkers(base, 12, seed=2)
    g, o, compared, diverged, observed, n_ex = run_cycle_lockstep(base, pos, n, blocks=2, steps=3, x0=0.5, n_c=1023)
    if not diverged:
        assert_same_state(g, o, base, observed)
