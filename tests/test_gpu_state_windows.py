"""Per-state energy histograms on the GPU (regc_set_state_windows,
regc_state_histograms): the observations of each state (Sec. II.B), binned in
a window of that state's own with an underflow and an overflow bin.

* Lock-step with the oracle on the 16-replica fcc(100) workload: every count
  equal, except observations whose energy lies within the energy tolerance of
  a bin edge (the GPU's running energy is exact fixed point, the oracle's
  FP64), which may sit in the neighbouring bin; every row sums to omega.
* Windows centred by the library sit at mean - n_bins e_bin / 2 of each
  state's observed energies, on the 2^-30 grid.
* A checkpoint carries the windows and their counts (a handle without windows
  refuses it); a batch fills them exactly as stepping its members alone.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Batch, Regc
from paper_1908_11118_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def test_state_windows_lockstep_with_oracle():
    p = W.fcc100_small()
    rng = np.random.default_rng(3)
    pos, n = W.initial_walkers(p, rng.integers(5, 25, p.S), seed=7)
    n_bins, e_bin = 4096, 0.0625
    e_lo = -200.0 + 2.5 * np.arange(p.S)          # exact on the 2^-30 grid
    g = Regc(p)
    g.set_walkers(pos, n)
    g.set_state_windows(n_bins, e_bin, e_lo)
    o = O.Oracle(p, pos=pos, n=n)
    o.set_state_windows(n_bins, e_bin, e_lo)
    near = 0
    for block in range(6):
        g.sweep(10)
        for _ in range(10):
            o.sweeps(1)
            x = (o.energy - e_lo[o.state_of_walker]) / e_bin
            tol = 1e-4 * np.maximum(1.0, np.abs(o.energy)) / e_bin
            near += int(np.sum(np.abs(x - np.round(x)) <= tol))
        g.exchange()
        o.exchange()
    gp, gn, ge, gs = g.get_walkers()
    assert np.array_equal(gn, o.n) and np.array_equal(gs, o.state_of_walker), "chains parted at a near tie"
    hE, lo, eb = g.state_histograms()
    assert eb == e_bin and np.array_equal(lo, e_lo)
    assert np.array_equal(hE.sum(axis=1), g.histograms()["omega"])
    assert np.array_equal(hE.sum(axis=1), o.omega)
    assert np.abs(hE - o.hE).sum() <= 2 * near
    assert hE[:, 1:-1].sum() > 0.9 * hE.sum()      # the windows hold the energies


def test_centred_windows_and_reset():
    p = W.fcc100_small(L=2, M=2)
    pos, n = W.initial_walkers(p, 10, seed=2)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.run(40)
    h = g.histograms()
    mean = h["moments"][:, 2] / h["omega"]
    g.set_state_windows(256, 0.1, None)
    hE, lo, eb = g.state_histograms()
    assert hE.sum() == 0                            # zeroed when set
    grid = 2.0 ** 30
    assert eb == np.round(0.1 * grid) / grid
    np.testing.assert_array_equal(lo, np.round((mean - 128 * eb) * grid) / grid)
    g.run(20)
    hE, _, _ = g.state_histograms()
    assert hE.sum() == 20 * p.S
    g.reset_histograms()
    assert g.state_histograms()[0].sum() == 0
    g.set_state_windows(0, 0.1, None)               # switched off
    with pytest.raises(Exception):
        g.state_histograms()
    with pytest.raises(Exception):
        g.set_state_windows(16, 0.0, None)


def test_checkpoint_carries_state_windows():
    p = W.fcc100_small(seed=3)
    pos, n = W.initial_walkers(p, 12, seed=2)
    e_lo = -50.0 + np.arange(p.S)

    def make():
        g = Regc(p)
        g.set_walkers(pos, n)
        g.set_state_windows(512, 0.125, e_lo)
        return g

    g = make()
    g.run(30)
    ck = g.checkpoint()
    g.run(30)
    want = g.state_histograms()[0]
    h = make()
    h.restore(ck)
    h.run(30)
    assert np.array_equal(h.state_histograms()[0], want)
    bare = Regc(p)
    with pytest.raises(Exception):
        bare.restore(ck)


def test_batch_fills_state_windows_like_members_alone():
    ps = [W.fcc100_small(L=2, M=2, seed=5), W.fcc100_small(L=2, M=3, nmax=24, seed=6)]
    alone, members = [], []
    for k, p in enumerate(ps):
        pos, n = W.initial_walkers(p, 6 + k, seed=k)
        for lst in (alone, members):
            g = Regc(p)
            g.set_walkers(pos, n)
            g.set_state_windows(300, 0.25, -40.0 + 0.5 * np.arange(p.S))
            lst.append(g)
    b = Batch(members, sweeps_per_step=5)
    b.run(4)
    b.sync()
    for g in alone:
        for _ in range(4):
            g.sweep(5)
            g.exchange()
    for a, m in zip(alone, members):
        assert np.array_equal(a.state_histograms()[0], m.state_histograms()[0])
        assert np.array_equal(a.get_walkers()[1], m.get_walkers()[1])
