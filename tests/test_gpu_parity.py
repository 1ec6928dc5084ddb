"""GPU parity: the CUDA sampler against the FP64 oracle, move by move.

Every test calls the library through its C ABI (via the ctypes binding) and
compares with the oracle on identical seeded inputs:
  * traces of every trial move (type, particle, status, energy change within
    1e-5 of max(|dE|, sum |phi|), acceptance; decisions may differ only at a
    near-tie, after which the walker is no longer compared);
  * final configurations bit for bit, N, energies, state labels after
    replica exchanges, histograms and counters;
  * the running energy against a from-scratch recompute (exactly zero drift);
  * edge cases: empty and full walkers, Nmax = 1, ragged Nmax, more than 32
    moves per sweep, fewer than three cells along an axis, a periodic cube
    without surface, a single state, displacement-only and GC-only move sets;
  * the 1024-replica, Nmax-512 fcc(111) workload in the launch configuration
    the benchmark times.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from paper_1908_11118_gb300 import Regc
from paper_1908_11118_gb300 import build as B
from parity import compare_traces

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def beta_max(p):
    return 1.0 / float(np.min(p.kT))


def run_lockstep(p, pos, n, blocks, sweeps, exchange=True, min_moves=1):
    """Run GPU and oracle side by side; compare each block.  Returns
    (gpu, oracle, compared, diverged, observed) where observed lists the
    oracle's energy at every per-sweep observation."""
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    e_g = g.get_walkers()[2]
    tol = 1e-5 * np.maximum(1.0, np.abs(o.energy)) + 1e-6
    assert np.all(np.abs(e_g - o.energy) <= tol * 10), "initial energies differ"
    compared, diverged, observed = 0, [], []
    for b in range(blocks):
        e0 = o.energy.copy()
        tg = g.sweep_traced(sweeps)
        to = o.sweeps(sweeps, trace=True)
        # energy after each sweep, rebuilt from the accepted moves
        de = np.where(to["accepted"] == 1, to["dE"], 0.0).sum(axis=2)
        observed.append(e0[:, None] + np.cumsum(de, axis=1))
        c, d = compare_traces(tg, to, beta_max(p))
        compared += c
        if d:
            diverged = d
            break
        if exchange:
            g.exchange()
            o.exchange()
    assert compared >= min_moves
    return g, o, compared, diverged, np.concatenate(observed, axis=1).ravel()


def assert_same_state(g, o, p, observed):
    pos, n, e, sow = g.get_walkers()
    assert np.array_equal(n, o.n)
    assert np.array_equal(sow, o.state_of_walker)
    for w in range(p.S):
        assert np.array_equal(pos[w, :n[w]], o.pos[w, :n[w]].astype(np.float32)), "walker %d positions" % w
    scale = np.maximum(1.0, np.abs(o.energy))
    assert np.all(np.abs(e - o.energy) <= 1e-4 * scale)
    h = g.histograms()
    assert np.array_equal(h["hN"], o.hN)
    assert np.array_equal(h["omega"], o.omega)
    np.testing.assert_allclose(h["moments"][:, :2], o.moments[:, :2], rtol=1e-12)
    np.testing.assert_allclose(h["moments"][:, 2], o.moments[:, 2], rtol=1e-5, atol=1e-3)
    # pooled (N, E) histogram: a sample may land in the neighbouring E bin only
    # when its energy lies within the energy tolerance of a bin edge
    assert int(h["hNE"].sum()) + int(h["e_out"].sum()) == int(o.hNE.sum()) + int(o.e_out.sum())
    x = (observed - p.e_lo) / p.e_bin
    near_edge = np.abs(x - np.round(x)) * p.e_bin <= 1e-4 * np.maximum(1.0, np.abs(observed))
    mism = np.abs(h["hNE"] - o.hNE).sum() + np.abs(h["e_out"] - o.e_out).sum()
    assert mism <= 2 * int(near_edge.sum()), (mism, int(near_edge.sum()))
    mv, ex, pr = g.counters()
    assert np.array_equal(mv, o.counts)
    assert np.array_equal(ex, o.ex_counts)


def test_lockstep_fcc100_16_replicas():
    p = W.fcc100_small()
    rng = np.random.default_rng(0)
    pos, n = W.initial_walkers(p, rng.integers(0, 25, p.S), seed=1)
    g, o, compared, diverged, observed = run_lockstep(p, pos, n, blocks=8, sweeps=10, min_moves=p.S * 20 * 10)
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0


def dense_slab_long_columns():
    """4-layer fcc(100) slab of spacing 1.0 under a 5.5-high gas region: up to
    80 surface images per column, so a column spans three 32-slot batches."""
    xyz, lx, ly, ztop = W.fcc100_slab(6, 6, 4, 1.0)
    eps, sig = W._pair_tables(1.0, 1.0, 1.5, 0.9)
    return W.Problem(
        n_types=2, eps=eps, sigma=sig, rc=2.5, Lx=lx, Ly=ly, Lz=ztop + 6.0, periodic_z=0,
        z_lo=ztop + 0.5, z_hi=ztop + 6.0, surf_xyz=xyz, surf_type=np.ones(len(xyz), np.int32),
        kT=np.array([0.9, 1.4]), mu=np.array([-4.0, -2.5]), lambda0=1.0, nmax=48, moves_per_sweep=20,
        max_disp=0.25, p_disp=1.0 / 3.0, seed=5, e_lo=-700.0, e_bin=0.1, n_e_bins=8000, name="dense_slab")


EDGE_CASES = {
    "dense_slab_long_columns": lambda: (dense_slab_long_columns(), 10),
    "empty_walkers": lambda: (W.fcc100_small(), 0),
    "nmax_1": lambda: (W.fcc100_small(nmax=1), "half"),
    "ragged_nmax_37_full": lambda: (W.fcc100_small(L=1, M=1, nmax=37).replace(mu=np.array([-1.0])), "full"),
    "dense_nmax_64": lambda: (W.fcc100_small(L=2, M=2, nmax=64), 55),
    "moves_45_p_disp_08": lambda: (W.fcc100_small(L=2, M=3).replace(moves_per_sweep=45, p_disp=0.8), 12),
    "displacement_only": lambda: (W.fcc100_small(L=2, M=2).replace(p_disp=1.0), 20),
    "gc_only": lambda: (W.fcc100_small(L=2, M=2).replace(p_disp=0.0), 10),
    "one_cell_per_axis": lambda: (W.tiny_box(nmax=6, rc=1.5, kT=(0.8, 1.3), mu=(-3.0, -2.0)), 3),
    "periodic_cube_no_surface": lambda: (W.Problem(
        n_types=1, eps=np.diag([1.0, 0.0, 0.0, 0.0]), sigma=np.ones((4, 4)), rc=2.5, Lx=7.6, Ly=7.6, Lz=7.6, periodic_z=1, z_lo=0.0, z_hi=7.6,
        surf_xyz=np.zeros((0, 3)), surf_type=np.zeros(0, np.int32), kT=np.array([0.9, 1.4]),
        mu=np.array([-4.0, -2.5]), lambda0=1.0, nmax=40, moves_per_sweep=45, max_disp=0.3,
        p_disp=0.5, seed=3, e_lo=-400.0, e_bin=0.1, n_e_bins=8000), 20),
}


@pytest.mark.parametrize("case", sorted(EDGE_CASES))
def test_lockstep_edge_cases(case):
    p, n0 = EDGE_CASES[case]()
    if n0 == "full":
        n0 = p.nmax
    elif n0 == "half":
        n0 = np.arange(p.S) % 2
    pos, n = W.initial_walkers(p, n0, seed=7, min_dist=0.85)
    g, o, compared, diverged, observed = run_lockstep(p, pos, n, blocks=4, sweeps=5)
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0


def test_production_kernel_matches_traced_kernel():
    """The untraced kernel (the one regc_sweep runs) makes the same moves."""
    p = W.fcc100_small()
    pos, n = W.initial_walkers(p, 15, seed=4)
    a, b = Regc(p), Regc(p)
    a.set_walkers(pos, n)
    b.set_walkers(pos, n)
    for _ in range(3):
        a.sweep(10)
        a.exchange()
        b.sweep_traced(10)
        b.exchange()
    sa, sb = a.get_walkers(), b.get_walkers()
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    assert np.array_equal(a.histograms()["hNE"], b.histograms()["hNE"])


@pytest.mark.parametrize("warps", [2, 4])
def test_speculative_walkers_make_the_sequential_chain(warps, monkeypatch):
    """Two and four warps per walker (moves evaluated speculatively, committed
    in order) end in the state of one warp per walker, bit for bit, on the
    fcc(111) slab with 256 replicas (the launch shape is picked at handle
    creation; REGC_WARPS_PER_WALKER forces it)."""
    p = W.fcc111_paper_scale(L=8)
    rng = np.random.default_rng(2)
    pos, n = W.lattice_walkers(p, rng.integers(0, p.nmax // 2 + 1, p.S), seed=2)
    monkeypatch.setenv("REGC_WARPS_PER_WALKER", "1")
    one = Regc(p)
    monkeypatch.setenv("REGC_WARPS_PER_WALKER", str(warps))
    spec = Regc(p)
    assert one.warps_per_walker() == 1 and spec.warps_per_walker() == warps
    for g in (one, spec):
        g.set_walkers(pos, n)
        for _ in range(3):
            g.sweep(10)
            g.exchange()
    for x, y in zip(one.get_walkers(), spec.get_walkers()):
        assert np.array_equal(x, y)
    assert np.array_equal(one.histograms()["hNE"], spec.histograms()["hNE"])
    assert spec.check_energy() == 0.0


def test_full_size_fcc111_1024_replicas():
    """The 1024-replica Nmax-512 workload in the benchmark's launch
    configuration: ten traced sweeps of every walker from the benchmark's
    initial state, every move compared with the oracle; every walker that did
    not part from the oracle at a near tie ends in the oracle's state
    (positions bit for bit, N, energy); then one exchange attempt (state labels
    equal when no walker parted); the untraced kernel over the same sweeps and
    exchange reaches the same state as the traced one."""
    p = W.fcc111_paper_scale()
    rng = np.random.default_rng(0)
    pos, n = W.lattice_walkers(p, rng.integers(0, p.nmax // 2 + 1, p.S), seed=0)
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    tg = g.sweep_traced(10)
    to = o.sweeps(10, trace=True)
    compared, diverged = compare_traces(tg, to, beta_max(p))
    assert compared >= 0.99 * p.S * 10 * p.moves_per_sweep
    assert len(diverged) <= p.S // 100
    gp, gn, ge, _ = g.get_walkers()
    same = np.setdiff1d(np.arange(p.S), diverged)
    assert np.array_equal(gn[same], o.n[same])
    for w in same:
        assert np.array_equal(gp[w, :gn[w]], o.pos[w, :gn[w]].astype(np.float32)), "walker %d positions" % w
    scale = np.maximum(1.0, np.abs(o.energy[same]))
    assert np.all(np.abs(ge[same] - o.energy[same]) <= 1e-4 * scale)
    assert g.check_energy() == 0.0
    g.exchange()
    o.exchange()
    if not diverged:
        assert np.array_equal(g.get_walkers()[3], o.state_of_walker)
    prod = Regc(p)
    prod.set_walkers(pos, n)
    prod.sweep(10)
    prod.exchange()
    for x, y in zip(prod.get_walkers(), g.get_walkers()):
        assert np.array_equal(x, y)


def test_set_walkers_rejects_overlaps():
    p = W.fcc100_small(L=1, M=1)
    pos = np.zeros((1, p.nmax, 3))
    pos[0, 0] = [1.0, 1.0, 5.0]
    pos[0, 1] = [1.05, 1.0, 5.0]
    g = Regc(p)
    with pytest.raises(Exception):
        g.set_walkers(pos, np.array([2], np.int32))
    pos[0, 1] = [2.5, 1.0, 5.0]
    g.set_walkers(pos, np.array([2], np.int32))
    assert g.get_walkers()[1][0] == 2


def test_torch_stream_is_used():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    p = W.fcc100_small(L=2, M=2)
    pos, n = W.initial_walkers(p, 5, seed=2)
    g = Regc(p, stream=s)
    g.set_walkers(pos, n)
    g.sweep(5)
    g.exchange()
    ref = Regc(p)
    ref.set_walkers(pos, n)
    ref.sweep(5)
    ref.exchange()
    for x, y in zip(g.get_walkers(), ref.get_walkers()):
        assert np.array_equal(x, y)


def test_walker_io_round_trip_and_checks():
    """Walker state goes in and out bit for bit (entries beyond N are ignored on
    the way in); a coordinate outside the region or N out of range is refused."""
    p = W.fcc100_small(L=2, M=2)
    pos, n = W.initial_walkers(p, np.array([0, 3, 17, 32]), seed=9)
    pos = np.asarray(pos, np.float32).copy()
    pos[0, :] = 123.0              # beyond N = 0: ignored
    pos[1, 3:] = -5.0              # beyond N = 3: ignored
    g = Regc(p)
    g.set_walkers(pos, n, np.array([3, 2, 1, 0], np.int32))
    pg, ng, eg, sg = g.get_walkers()
    assert np.array_equal(ng, n) and np.array_equal(sg, [3, 2, 1, 0])
    for w in range(p.S):
        assert np.array_equal(pg[w, :n[w]], pos[w, :n[w]])
    o = O.Oracle(p, pos=pos, n=n)
    assert np.all(np.abs(eg - o.energy) <= 1e-5 * np.maximum(1.0, np.abs(o.energy)))
    bad = pos.copy()
    bad[2, 5, 2] = p.z_lo - 0.5    # below the region
    with pytest.raises(Exception):
        g.set_walkers(bad, n)
    assert np.all(g.get_walkers()[1] == 0)       # left empty
    with pytest.raises(Exception):
        g.set_walkers(pos, np.array([0, 3, 17, p.nmax + 1], np.int32))
    g.set_walkers(pos, n)
    assert np.array_equal(g.get_walkers()[1], n)
    assert g.check_energy() == 0.0
