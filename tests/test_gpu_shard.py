"""A grid split over processes (regc_set_shard, regc_get_walker_ne,
regc_set_walker_ne; paper_1908_11118_gb300/shard.py) on one GPU: two handles
of the 1024-replica workload, each stepping half of the walkers, exchange
through the all-gather of (N, E) -- here an in-process gather -- and must end
in the state of one handle stepping all walkers, walker for walker and bit for
bit, with histograms that sum to its own.  The ranks' kernels never wait on
one another: the only meeting point is the host-side gather."""
import numpy as np
import pytest

import workloads as W
from paper_1908_11118_gb300 import RegcError, shard
from paper_1908_11118_gb300 import build as B
from paper_1908_11118_gb300.regc import Regc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _exchange_all(engines):
    """One sharded exchange attempt on every engine, the gather being the
    list of every engine's item."""
    items = []
    for g in engines:
        b, e = g.shard
        items.append(((b, e), g.walker_ne(b, e)))
    for g in engines:
        shard.exchange(g, lambda item: items)


def _start(p, world):
    rng = np.random.default_rng(0)
    pos, n = W.lattice_walkers(p, rng.integers(0, p.nmax // 2 + 1, p.S), seed=0)
    full = Regc(p)
    full.set_walkers(pos, n)
    parts = []
    for r in range(world):
        g = Regc(p)
        g.set_walkers(pos, n)
        g.set_shard(*shard.shard_range(p.S, r, world))
        parts.append(g)
    return full, parts


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_grid_matches_one_handle(world):
    p = W.fcc111_paper_scale()
    full, parts = _start(p, world)
    for _ in range(4):
        full.sweep(10)
        full.exchange()
        for g in parts:
            g.sweep(10)
        _exchange_all(parts)
    fp, fn, fe, fs = full.get_walkers()
    hsum = {}
    for g in parts:
        b, e = g.shard
        gp, gn, ge, gs = g.get_walkers()
        assert np.array_equal(gs, fs)                       # the same state labels everywhere
        assert np.array_equal(gn[b:e], fn[b:e])
        assert np.array_equal(ge[b:e], fe[b:e])
        assert np.array_equal(gp[b:e], fp[b:e])
        assert g.check_energy() == 0.0                      # the shard's own walkers
        h = g.histograms()
        for k in ("hN", "hNE", "omega"):
            hsum[k] = hsum.get(k, 0) + h[k]
    hf = full.histograms()
    for k in ("hN", "hNE", "omega"):
        assert np.array_equal(hsum[k], hf[k]), k
    assert not np.array_equal(fs, np.arange(p.S))           # swaps were accepted


def test_walker_ne_round_trip_and_refusals():
    p = W.fcc100_small()
    full, (g0, g1) = _start(p, 2)
    full.sweep(5)
    n, nb, e = full.walker_ne(0, p.S)
    assert nb is None
    assert np.array_equal(n, full.get_walkers()[1])
    assert np.allclose(e * 2.0 ** -30, full.get_walkers()[2], rtol=0, atol=1e-9)
    g0.set_walker_ne(8, n[8:], None, e[8:])
    n2, _, e2 = g0.walker_ne(8, 16)
    assert np.array_equal(n2, n[8:]) and np.array_equal(e2, e[8:])
    bad = n[8:].copy()
    bad[0] = p.nmax + 1
    with pytest.raises(RegcError):
        g0.set_walker_ne(8, bad, None, e[8:])
    for args in ((0, 0), (-1, 4), (4, p.S + 1), (5, 3)):
        with pytest.raises(RegcError):
            g0.set_shard(*args)
    # calls that need every walker's configuration refuse a proper shard
    with pytest.raises(RegcError):
        g0.sweep_traced(1)
    with pytest.raises(RegcError):
        g0.cycle(2, 0.99, 10)
    with pytest.raises(RegcError):
        g0.md(2, 0.001, 0.1)
    g0.set_shard(0, p.S)                                    # the whole grid again
    g0.sweep_traced(1)


def test_sharded_two_species_grid_matches_one_handle():
    """Two grand-canonical species (N_B carried with N and E, the fifth
    exchange direction along mu_C): three sharded handles against one."""
    p = W.two_gas_small(seed=5)
    rng = np.random.default_rng(5)
    pos, n, nbv = W.two_gas_initial(p, rng.integers(0, 6, p.S), rng.integers(0, 6, p.S), seed=5)
    full = Regc(p)
    full.set_walkers(pos, n, nb=nbv)
    parts = []
    for r in range(3):
        g = Regc(p)
        g.set_walkers(pos, n, nb=nbv)
        g.set_shard(*shard.shard_range(p.S, r, 3))
        parts.append(g)
    for _ in range(6):
        full.sweep(10)
        full.exchange()
        for g in parts:
            g.sweep(10)
        _exchange_all(parts)
    fp, fn, fe, fs = full.get_walkers()
    fnb = full.walker_ne(0, p.S)[1]
    for g in parts:
        b, e = g.shard
        gp, gn, ge, gs = g.get_walkers()
        assert np.array_equal(gs, fs)
        assert np.array_equal(gn[b:e], fn[b:e]) and np.array_equal(ge[b:e], fe[b:e])
        assert np.array_equal(g.walker_ne(b, e)[1], fnb[b:e])
        assert np.array_equal(gp[b:e], fp[b:e])
