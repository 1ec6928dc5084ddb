"""GPU parity in a sheared cell: the paper's own 3 x 3 hexagonal fcc(111)
cell of the LJ surface of Sec. III.A (18 A atoms, coordinates in the cell
frame), against the FP64 oracle.

* From-scratch energies of seeded walkers.
* Sweeps and the REGC cycle in lock-step, move by move: the paper's 160
  replicas at x0 = 0.99, and a 16-replica grid with delayed acceptance.
* A short MD segment (positions, kinetic energies).
* Structure counts, including the 18 hollow sites whose lateral pair shells
  are known in closed form.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from oracle import structure as ST
from paper_1908_11118_gb300 import Regc
from paper_1908_11118_gb300 import build as B
from parity import compare_da_traces
from test_gpu_cycle import run_cycle_lockstep
from test_gpu_parity import assert_same_state, beta_max, run_lockstep
from test_gpu_structure import assert_same_samples, oracle_samples
from test_gpu_surrogate import sur_tol_of, theta_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def test_energies_match_oracle():
    p = W.lj_a18_hex_slab(L=2, M=4, nmax=96, seed=1)
    rng = np.random.default_rng(1)
    pos, n = W.lj_a18_initial(p, rng.integers(0, 80, p.S), seed=2)
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    e = g.get_walkers()[2]
    np.testing.assert_allclose(e, o.energy, rtol=1e-5, atol=1e-4)


def test_sweeps_lockstep():
    p = W.lj_a18_hex_slab(L=4, M=4, nmax=96, seed=3)
    rng = np.random.default_rng(4)
    pos, n = W.lj_a18_initial(p, rng.integers(0, 70, p.S), seed=5)
    g, o, compared, diverged, observed = run_lockstep(p, pos, n, blocks=6, sweeps=10, min_moves=p.S * 11 * 10 * 3)
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0


def test_paper_cycle_160_replicas_lockstep():
    p = W.lj_a18_hex_slab(nmax=128, seed=6)
    rng = np.random.default_rng(7)
    pos, n = W.lj_a18_initial(p, rng.integers(0, 60, p.S), seed=8)
    g, o, compared, diverged, observed, n_ex = run_cycle_lockstep(p, pos, n, blocks=2, steps=150, x0=0.99, n_c=10,
                                                                  min_moves=p.S * 10 * 150)
    assert len(diverged) <= 2
    if not diverged:
        assert_same_state(g, o, p, observed)
    assert g.check_energy() == 0.0


def test_delayed_acceptance_lockstep():
    p = W.lj_a18_hex_slab(L=4, M=4, nmax=96, seed=9)
    pos, n = W.lj_a18_initial(p, 30, seed=10)
    th = theta_of(4)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.surrogate_set(th)
    g.set_mode(True)
    o = O.Oracle(p, pos=pos, n=n, surrogate=th)
    beta = np.full(p.S, beta_max(p))
    for b in range(3):
        tg, _ = g.cycle_traced(20, 0.95, 10)
        to, _ = o.cycle(20, 0.95, 10, trace=True)
        c, x, d = compare_da_traces(tg, to, beta, sur_tol_of)
        if d:
            return
    pg, ng, _, sg = g.get_walkers()
    assert np.array_equal(ng, o.n) and np.array_equal(sg, o.state_of_walker)
    for w in range(p.S):
        assert np.array_equal(pg[w, :ng[w]], o.pos[w, :ng[w]].astype(np.float32))


def test_md_short_segment():
    p = W.lj_a18_hex_slab(L=2, M=2, nmax=64, seed=11)
    pos, n = W.lj_a18_initial(p, [5, 18, 30, 45], seed=12)
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    dt = 0.002 * 10.0          # time units of eV, A and u: about 2 fs steps are ~0.02
    kg = g.md(5, dt, 0.5)
    ko = o.md(5, dt, 0.5)
    pg, ng, eg, _ = g.get_walkers()
    L = np.array([p.Lx, p.Ly])
    for w in range(p.S):
        d = pg[w, :ng[w]] - o.pos[w, :ng[w]]
        d[:, :2] -= np.round(d[:, :2] / L) * L
        assert np.max(np.abs(d)) < 5e-5, w
    np.testing.assert_allclose(kg, ko, rtol=5e-4, atol=1e-5)
    np.testing.assert_allclose(eg, o.energy, rtol=1e-4, atol=1e-3)


def test_structure_counts_and_hollow_shells():
    p = W.lj_a18_hex_slab(L=2, M=2, nmax=64, seed=13)
    pos, n = W.lj_a18_initial(p, [18, 25, 40, 60], seed=14)
    xy = W.hex_hollow_sites(p)
    pos[0] = 0.0
    pos[0, :18, :2] = xy
    pos[0, :18, 2] = p.z_lo + 0.05
    pos[0] = W.f32(pos[0])
    n[0] = 18
    spec = {"n_z": 400, "dz": 0.12, "layers": [(p.z_lo, p.z_lo + 0.6), (p.z_lo + 0.6, p.z_lo + 2.0)],
            "n_r": 49, "dr": 0.1}
    g = Regc(p)
    g.set_walkers(pos, n)
    g.structure_init(spec["n_z"], spec["dz"], spec["layers"], spec["n_r"], spec["dr"], p.S)
    g.structure_sample()
    gs = g.structure_get()
    o = O.Oracle(p, pos=pos, n=n)
    assert_same_samples(gs, *oracle_samples(p, o, spec))
    a = p.Lx / 3.0
    want = np.zeros(49, np.int64)
    for d, z in ((a / math.sqrt(3.0), 3), (a, 6), (2.0 * a / math.sqrt(3.0), 3)):
        want[int(d / 0.1)] += 18 * z // 2
    assert np.array_equal(gs["pairs"][0, 0].astype(np.int64), want)
    with pytest.raises(Exception):     # beyond the inscribed radius of the sheared cell (4.975 A)
        g.structure_init(10, 0.5, [], 50, 0.1, p.S)
