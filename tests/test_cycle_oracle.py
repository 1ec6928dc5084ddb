"""Pins of the oracle's REGC cycle (Sec. II.A and Fig. 1: with probability x0
a particle exchange with the reservoir, else a replica-exchange attempt, then
canonical diffusion; Sec. III.A: x0 = 0.99, insertion and removal equally
likely, ten MC moves after each attempt).

* The schedule: the number of replica-exchange steps over many steps is
  binomial with p = 1 - x0; insertion and removal attempts are equally
  likely; each particle-exchange step costs every replica exactly one
  insertion or removal trial and each step exactly n_canonical displacement
  trials; the exchange numbers advance once per replica-exchange step.
* The sampling: the cycle keeps the grand-canonical distribution of the small
  box (brute-force <N> and <E> per state) and of the ideal gas (truncated
  Poisson <N>), the latter with replica exchange every other step.
* Planted mistakes: the two branches of the x0 choice swapped (2048), the
  canonical moves drawn from the mixed move set (4096), and the swap-rule
  mistakes 1 and 2 seen through the cycle.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from test_oracle_pins import ideal_lambda, small_box_problem, trunc_poisson, zscores
from test_md_oracle import expected_small_box


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def schedule_pin(mutation=0, n_steps=20000, x0=0.9, n_c=2):
    """Largest violation among the schedule's checks: binomial z-scores, and
    any exact count that is off (returned as inf)."""
    p = W.ideal_gas(W.fcc100_small(L=1, M=2, nmax=16, seed=3))
    o = O.Oracle(p, mutation=mutation)
    tr, n_ex = o.cycle(n_steps, x0, n_c, hist=False, trace=True)
    worst = abs(n_ex - (1 - x0) * n_steps) / math.sqrt(n_steps * x0 * (1 - x0))
    if o.e != n_ex:
        return math.inf
    re_steps = tr["type"][0, :, 0] == -1
    if int(re_steps.sum()) != n_ex or np.any((tr["type"][:, :, 0] == -1) != re_steps[None, :]):
        return math.inf                        # every replica sees the same choice
    if np.any(tr["status"][:, re_steps, 0] != 4):
        return math.inf
    n_gc = n_steps - n_ex
    for w in range(p.S):
        trials = o.counts[w, :, 0]
        if trials[1] + trials[2] != n_gc or trials[0] != n_c * n_steps:
            return math.inf
        worst = max(worst, abs(trials[1] - trials[2]) / math.sqrt(n_gc))
    if np.any(tr["type"][:, :, 1:] != 0):
        return math.inf                        # canonical moves are displacements
    return worst


def test_schedule():
    assert schedule_pin() < 4.5


def test_choice_follows_its_counter():
    """Step t exchanges replicas iff word 0 of Philox((t, 0, 0, 10)) is at
    least floor(x0 2^32); the moves of step t are the moves of sweep t."""
    p = W.fcc100_small(L=2, M=2, seed=5)
    pos, n = W.initial_walkers(p, 6, seed=1)
    o = O.Oracle(p, pos=pos, n=n)
    o.sweeps(3, hist=False)                    # the step counter continues the sweep counter
    x0 = 0.7
    tr, n_ex = o.cycle(200, x0, 3, hist=False, trace=True)
    key = (p.seed & 0xFFFFFFFF, p.seed >> 32)
    th = math.floor(x0 * 2 ** 32)
    want = np.array([O.philox4x32_10((t, 0, 0, 10), key)[0] >= th for t in range(3, 203)])
    assert np.array_equal(tr["type"][0, :, 0] == -1, want)
    assert n_ex == int(want.sum())


def test_x0_one_and_zero():
    p = W.fcc100_small(L=2, M=2, seed=6)
    o = O.Oracle(p)
    _, n_ex = o.cycle(50, 1.0, 2, hist=False)
    assert n_ex == 0
    _, n_ex = o.cycle(50, 0.0, 2, hist=False)
    assert n_ex == 50
    assert o.counts[:, 1:, 0].sum() == 50 * p.S      # GC trials only in the x0 = 1 steps
    with pytest.raises(ValueError):
        o.cycle(5, 1.5, 2)
    with pytest.raises(ValueError):
        o.cycle(5, 0.5, -1)


def test_no_canonical_moves_observes_particle_exchange_steps_only():
    """n_canonical = 0 (REGCMD: the canonical diffusion is MD): a replica is
    observed after its particle-exchange attempt; a replica-exchange step has
    no move and no observation."""
    p = W.fcc100_small(L=2, M=2, seed=7)
    o = O.Oracle(p)
    tr, n_ex = o.cycle(400, 0.7, 0, trace=True)
    assert tr.shape == (p.S, 400, 1)
    assert o.omega.sum() == p.S * (400 - n_ex)
    assert o.counts[:, 0, 0].sum() == 0                    # no displacement
    assert o.counts[:, 1:, 0].sum() == p.S * (400 - n_ex)


def small_box_cycle_pin(mutation=0, n_batches=16, steps=6000, x0=0.9, n_c=4):
    p = small_box_problem()
    o = O.Oracle(p, mutation=mutation)
    o.cycle(500, x0, n_c, hist=False)
    nv = np.arange(p.nmax + 1)
    nb, eb = np.zeros((n_batches, p.S)), np.zeros((n_batches, p.S))
    for b in range(n_batches):
        h0, m0, om0 = o.hN.copy(), o.moments.copy(), o.omega.copy()
        o.cycle(steps, x0, n_c)
        dh = o.hN - h0
        nb[b] = (dh @ nv) / np.maximum(dh.sum(axis=1), 1)
        eb[b] = (o.moments[:, 2] - m0[:, 2]) / np.maximum(o.omega - om0, 1)
    exp_n, exp_e, sd_n = expected_small_box(p)
    zn = zscores(nb, exp_n, sd_n, n_batches * steps)
    ze = zscores(eb, exp_e, np.ones(p.S), n_batches * steps)
    return float(max(np.max(np.abs(zn)), np.max(np.abs(ze))))


def test_small_box_brute_force():
    assert small_box_cycle_pin() < 4.5


def ideal_gas_cycle_pin(mutation=0, n_batches=16, steps=1500):
    """x0 = 0.5: a replica-exchange attempt every other step on average, one
    displacement after each, so that a wrong swap rule shows in <N>."""
    p = W.ideal_gas(W.fcc100_small())
    o = O.Oracle(p, mutation=mutation)
    nv = np.arange(p.nmax + 1)
    nb = np.zeros((n_batches, p.S))
    for b in range(n_batches):
        h0 = o.hN.copy()
        o.cycle(steps, 0.5, 1)
        dh = o.hN - h0
        nb[b] = (dh @ nv) / np.maximum(dh.sum(axis=1), 1)
    exp_mean, exp_sd = np.zeros(p.S), np.zeros(p.S)
    for s in range(p.S):
        pr = trunc_poisson(ideal_lambda(p, s), p.nmax)
        exp_mean[s] = pr @ nv
        exp_sd[s] = math.sqrt(pr @ nv ** 2 - exp_mean[s] ** 2)
    return float(np.max(np.abs(zscores(nb, exp_mean, exp_sd, n_batches * steps))))


def test_ideal_gas_with_frequent_exchange():
    assert ideal_gas_cycle_pin() < 4.5


def test_planted_branch_swap_is_detected():
    assert schedule_pin(mutation=2048) > 6.0


def test_planted_mixed_canonical_moves_are_detected():
    assert schedule_pin(mutation=4096) == math.inf


@pytest.mark.parametrize("bit", [1, 2])
def test_planted_swap_rule_mistakes_are_detected_through_the_cycle(bit):
    """A wrong swap rule (1: the sign of the mu term; 2: the Lambda factor
    dropped) biases <N> of the ideal gas under the cycle."""
    assert ideal_gas_cycle_pin(mutation=bit, n_batches=8, steps=1500) > 6.0
