"""GPU tests of the batch of uneven systems.

One batch step is defined as regc_sweep(h, sweeps_per_step) + regc_exchange(h)
on every member with the same Philox streams, so:
  * a batch (size-class persistent kernels, captured graph, autotuned shapes)
    leaves every member bit-identical -- positions, N, energies, state labels,
    histograms, moments and counters -- to stepping the members one by one;
  * every member's final state equals the FP64 oracle's for the same steps;
  * stepping a member on its own between batch steps is picked up;
  * members in delayed-acceptance mode run in classes of their own, with the
    same bit-for-bit equality; a member whose mode changed after the batch
    was made is refused; parameters changed on a member after the batch was
    made (per-state windows) are picked up.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Batch, Regc
from paper_1908_11118_gb300 import build as B

pytestmark = pytest.mark.gpu

SPS = 5   # sweeps per step


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def small_uneven(n=6):
    # Nmax 32..128, slabs 4..6 atoms on a side, gas 6..9 high: four size classes
    return W.uneven_batch(n_systems=n, L=2, M=2, seed=3, nmax_exp=(5, 7), side=(4, 6), height=(6.0, 9.0))


def members(ps, seed):
    hs, init = [], []
    for i, p in enumerate(ps):
        pos, n = W.uneven_initial(p, seed + i)
        h = Regc(p)
        h.set_walkers(pos, n)
        hs.append(h)
        init.append((pos, n))
    return hs, init


def steps_done(h):
    mv = h.counters()[0]
    return int(mv[0, :, 0].sum()) // (SPS * h.mps)


def assert_same(a, b):
    for x, y in zip(a.get_walkers(), b.get_walkers()):
        assert np.array_equal(x, y)
    ha, hb = a.histograms(), b.histograms()
    for k in ha:
        assert np.array_equal(ha[k], hb[k]), k
    (ma, ea, pa), (mb, eb, pb) = a.counters(), b.counters()
    assert np.array_equal(ma, mb) and np.array_equal(ea, eb)
    # pairs within rc of the committed moves and the surrogate counts do not
    # depend on the launch shape; candidates, rounds and evaluations do (the
    # batch runs one warp per walker, a handle alone may speculate with more)
    assert pa[0] == pb[0] and np.array_equal(pa[4:], pb[4:])
    assert a.check_energy() == 0.0


def test_batch_equals_members_stepped_one_by_one():
    ps = small_uneven()
    A, _ = members(ps, 11)
    Bs, _ = members(ps, 11)
    with Batch(A, sweeps_per_step=SPS) as bt:
        plan0 = bt.plan()
        assert len(plan0) >= 2 and sum(c["walkers"] for c in plan0) == sum(p.S for p in ps)
        bt.autotune(1)
        bt.run(3)
        bt.sync()
        plan = bt.plan()
        assert all(c["ms"] > 0 for c in plan)
    k = steps_done(A[0])
    assert k >= 4
    for h in Bs:
        for _ in range(k):
            h.sweep(SPS)
            h.exchange()
    for a, b in zip(A, Bs):
        assert steps_done(a) == k
        assert_same(a, b)


def test_batch_matches_oracle():
    ps = small_uneven(4)
    A, init = members(ps, 21)
    with Batch(A, sweeps_per_step=SPS) as bt:
        bt.run(4)
        bt.sync()
    for h, p, (pos, n) in zip(A, ps, init):
        o = O.Oracle(p, pos=pos, n=n)
        for _ in range(4):
            o.sweeps(SPS)
            o.exchange()
        pg, ng, eg, sg = h.get_walkers()
        assert np.array_equal(ng, o.n) and np.array_equal(sg, o.state_of_walker)
        for w in range(p.S):
            assert np.array_equal(pg[w, :ng[w]], o.pos[w, :ng[w]].astype(np.float32))
        assert np.all(np.abs(eg - o.energy) <= 1e-4 * np.maximum(1.0, np.abs(o.energy)))
        assert np.array_equal(h.histograms()["hN"], o.hN)


def test_member_stepped_alone_between_batch_steps():
    ps = small_uneven(3)
    A, _ = members(ps, 31)
    Bs, _ = members(ps, 31)
    with Batch(A, sweeps_per_step=SPS) as bt:
        bt.run(1)
        bt.sync()
        A[1].sweep(3)
        A[1].exchange()
        A[1].get_walkers()          # synchronises the member's stream
        bt.run(2)
        bt.sync()
    for i, h in enumerate(Bs):
        h.sweep(SPS)
        h.exchange()
        if i == 1:
            h.sweep(3)
            h.exchange()
        for _ in range(2):
            h.sweep(SPS)
            h.exchange()
    for a, b in zip(A, Bs):
        assert_same(a, b)


def test_batch_with_delayed_acceptance_members_equals_one_by_one():
    """Members sampling with delayed acceptance (each with its own network)
    run in size classes of their own (the delayed-acceptance instantiation of
    the persistent kernel) next to plain members, and every member ends
    bit-identical to stepping it alone, surrogate counters included."""
    ps = small_uneven(4)
    A, _ = members(ps, 41)
    Bs, _ = members(ps, 41)
    for hs in (A, Bs):
        for i in (0, 2):
            hs[i].surrogate_init(seed=1 + i)
            hs[i].set_mode(True)
    with Batch(A, sweeps_per_step=SPS) as bt:
        plan = bt.plan()
        assert len(plan) >= 3
        bt.autotune(1)
        bt.run(3)
        bt.sync()
    k = steps_done(A[0])
    for h in Bs:
        for _ in range(k):
            h.sweep(SPS)
            h.exchange()
    for a, b in zip(A, Bs):
        assert_same(a, b)
    assert A[0].counters()[2][4] > 0              # stage-1 evaluations happened


def test_batch_refuses_a_member_whose_mode_changed():
    ps = small_uneven(2)
    A, _ = members(ps, 43)
    A[0].surrogate_init(seed=1)
    A[0].set_mode(True)
    with Batch(A, sweeps_per_step=SPS) as bt:
        bt.run(1)
        bt.sync()
        A[0].set_mode(False)
        with pytest.raises(Exception):
            bt.run(1)
        A[0].set_mode(True)
        bt.run(1)
        bt.sync()


def test_batch_picks_up_state_windows_set_after_it_was_made():
    """Parameters changed on a member after the batch was made (here its
    per-state energy windows) are uploaded before the next batch step."""
    ps = small_uneven(3)
    A, _ = members(ps, 51)
    Bs, _ = members(ps, 51)
    with Batch(A, sweeps_per_step=SPS) as bt:
        bt.run(1)
        bt.sync()
        for h in A:
            h.set_state_windows(64, 0.5, None)
            h.reset_histograms()
        bt.run(2)
        bt.sync()
    for h in Bs:
        h.sweep(SPS)
        h.exchange()
        h.set_state_windows(64, 0.5, None)
        h.reset_histograms()
        for _ in range(2):
            h.sweep(SPS)
            h.exchange()
    for a, b in zip(A, Bs):
        ha, hb = a.state_histograms(), b.state_histograms()
        assert ha[0].sum() > 0
        for x, y in zip(ha, hb):
            assert np.array_equal(x, y)
        assert_same(a, b)
