"""The exchange protocol of a grid split over processes (paper_1908_11118_gb300
/shard.py) on two and three CPU ranks (gloo), with the FP64 oracle as each rank's
engine: every rank sweeps only its own walkers, all-gathers (N, E) before each
exchange attempt (Sec. II.A.2, Eq. Pacc) and runs the same exchange.  The run
must be the single-process run walker for walker: the owned walkers'
positions, N and energies bit for bit, the same state labels on every rank,
and histograms that sum over the ranks to the single run's."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SWEEPS = 40


class OracleEngine:
    """The oracle behind the engine interface shard.py drives."""

    def __init__(self, o, shard):
        self.o = o
        self.shard = shard

    def sweep(self, k):
        self.o.sweeps(k, hist=True, walkers=self.shard)

    def walker_ne(self, b, e):
        return self.o.n[b:e].copy(), None, self.o.energy[b:e].copy()

    def set_walker_ne(self, b, n, nb, e):
        self.o.n[b:b + len(n)] = n
        self.o.energy[b:b + len(n)] = e

    def exchange(self):
        self.o.exchange()


def _problem_and_walkers():
    import workloads as W
    p = W.fcc100_small(seed=0)
    rng = np.random.default_rng(3)
    pos, n = W.lattice_walkers(p, rng.integers(0, p.nmax // 2 + 1, p.S), seed=3)
    return p, pos, n


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out, planted):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1908_11118_gb300 import shard
    p, pos, n = _problem_and_walkers()
    b, e = shard.shard_range(p.S, rank, world)
    o = O.Oracle(p, pos=pos, n=n, n_threads=1)
    eng = OracleEngine(o, (b, e))
    gather = shard.torch_gather()
    if planted:
        # a planted protocol mistake: exchange on stale (N, E) of the other range
        done = 0
        while done < SWEEPS:
            eng.sweep(10)
            done += 10
            eng.exchange()
    else:
        shard.run(eng, gather, SWEEPS, exchange_every=10)
    hist = shard.reduce_histograms({"hN": o.hN, "hNE": o.hNE, "omega": o.omega, "moments": o.moments}, gather)
    out[rank] = {"range": (b, e), "pos": o.pos[b:e].copy(), "n": o.n[b:e].copy(), "energy": o.energy[b:e].copy(),
                 "sow": o.state_of_walker.copy(), "hist": hist}
    dist.destroy_process_group()


def _run_ranks(planted, world=2):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out, planted), nprocs=world, join=True)
    return [out[r] for r in range(world)]


def _single_run():
    from oracle import oracle as O
    O.build()
    p, pos, n = _problem_and_walkers()
    o = O.Oracle(p, pos=pos, n=n, n_threads=1)
    o.run(SWEEPS, exchange_every=10)
    return o


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_grid_is_the_single_process_run(world):
    ref = _single_run()
    ranks = _run_ranks(planted=False, world=world)
    assert [r["range"] for r in ranks] == ([(0, 8), (8, 16)] if world == 2 else [(0, 5), (5, 10), (10, 16)])
    for r in ranks:
        b, e = r["range"]
        assert np.array_equal(r["sow"], ref.state_of_walker)
        assert np.array_equal(r["n"], ref.n[b:e])
        assert np.array_equal(r["energy"], ref.energy[b:e])
        assert np.array_equal(r["pos"], ref.pos[b:e])
        h = r["hist"]
        assert np.array_equal(h["hN"], ref.hN)
        assert np.array_equal(h["hNE"], ref.hNE)
        assert np.array_equal(h["omega"], ref.omega)
        np.testing.assert_allclose(h["moments"], ref.moments, rtol=1e-12, atol=1e-9)
    # the exchange moved labels: the test exercises accepted swaps
    assert not np.array_equal(ref.state_of_walker, np.arange(ref.p.S))


def test_exchange_on_stale_energies_is_caught():
    ref = _single_run()
    ranks = _run_ranks(planted=True)
    assert any(not np.array_equal(r["sow"], ref.state_of_walker) for r in ranks)


def test_shard_ranges_cover_the_grid():
    from paper_1908_11118_gb300 import shard
    for S, world in ((16, 2), (1024, 3), (4096, 8), (5, 5)):
        rs = [shard.shard_range(S, r, world) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == S
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        assert max(e - b for b, e in rs) - min(e - b for b, e in rs) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(4, 4, 4)
