"""GPU parity of the structural observables (regc_structure_*: Sec. III.A
"Structural properties", the axial distribution rho(z) in 0.12 A slabs and the
lateral RDF g_xy(r) of adsorbate layers; Sec. II.B, Eq. avegr, their MBAR
averages per phase) against the FP64 oracle.

* Per-sample counts (slabs, layer populations, pair counts) equal to the
  oracle's on seeded LJ A18 walkers, including the honeycomb of hollow sites
  whose pair shells are known in closed form.  The oracle decides bins in FP64,
  the GPU in binary32: a count may differ only by an item within binary32
  rounding of a bin edge landing in the neighbouring bin (the oracle lists
  those items; their number is bounded).
* The paper's run in lock-step with the oracle (160 replicas, x0 = 0.99, a
  sample every 100 steps): the same samples, then MBAR averages per phase at
  sampled and unsampled states within FP64 tolerance of the oracle's.
* Properties of the reweighted averages at any size: p sums to 1 over the
  phases, rho integrates to N_B when the slabs cover the zone.
* aiAT@REGC (Eq. aiTherm): the lowest sampled energy per composition and the
  stable composition per chemical potential against the oracle's, and the
  configuration kept for a composition.
* Store limits and argument checks.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import aiat as AI
from oracle import oracle as O
from oracle import structure as ST
from paper_1908_11118_gb300 import Regc
from paper_1908_11118_gb300 import build as B
from test_structure_oracle import hollow_sites

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def spec_of(p):
    return {"n_z": 400, "dz": 0.12,
            "layers": [(p.z_lo, p.z_lo + 0.6), (p.z_lo + 0.6, p.z_lo + 1.6), (p.z_lo + 1.6, p.z_lo + 2.6)],
            "n_r": 57, "dr": 0.1}


def init_store(g, spec, capacity):
    g.structure_init(spec["n_z"], spec["dz"], spec["layers"], spec["n_r"], spec["dr"], capacity)


def assert_same_samples(gs, os_, edges, e_tol=1e-4):
    """The GPU's samples against the oracle's: states, N_B and layer
    populations equal; slab and pair counts equal except items within binary32
    rounding of a bin edge (the oracle decides bins in FP64), which may sit in
    the neighbouring bin; energies within e_tol."""
    assert np.array_equal(gs["state"], os_["state"])
    assert np.array_equal(gs["N"], os_["N"])
    assert np.array_equal(gs["pop"].astype(np.int64), os_["pop"])
    bad, moved = ST.edge_moves(gs, os_, edges)
    n_items = int(os_["rho"].sum() + os_["pairs"].sum())
    n_edge = sum(len(e) for e in edges)
    assert bad == 0, "%d counts differ beyond the near-edge items (%d near an edge, %d moved)" % (bad, n_edge, moved)
    assert moved <= n_edge <= max(4, 1e-3 * n_items)
    assert np.all(np.abs(gs["E"] - os_["E"]) <= e_tol * np.maximum(1.0, np.abs(os_["E"])))
    return moved


def oracle_samples(p, o, spec):
    """The oracle's samples of the walkers it holds, and their near-edge items."""
    edges = []
    return ST.structure_of_walkers(p, o.pos, o.n, o.state_of_walker, o.energy, spec, edges=edges), edges


def test_sample_counts_match_oracle():
    p = W.lj_a18_slab(L=4, M=4, nmax=128, seed=2)
    rng = np.random.default_rng(3)
    pos, n = W.lj_a18_initial(p, rng.integers(0, 110, p.S), seed=4)
    # walker 0: the honeycomb of all 36 hollow sites, just above the floor
    xy, _ = hollow_sites(p)
    pos[0] = 0.0
    pos[0, :36, :2] = xy
    pos[0, :36, 2] = p.z_lo + 0.05
    pos[0] = W.f32(pos[0])
    n[0] = 36
    g = Regc(p)
    g.set_walkers(pos, n)
    spec = spec_of(p)
    init_store(g, spec, 4 * p.S)
    g.structure_sample()
    gs = g.structure_get()
    o = O.Oracle(p, pos=pos, n=n)
    os_, edges = oracle_samples(p, o, spec)
    assert_same_samples(gs, os_, edges)
    assert gs["pairs"][0, 0].sum() == 54 + 108 + 54       # the honeycomb's three shells within 5.7 A
    assert gs["rho"][0, 0] == 36


def run_lockstep_with_samples(p, pos, n, blocks, steps, x0, n_c, spec):
    g = Regc(p)
    g.set_walkers(pos, n)
    init_store(g, spec, blocks * p.S)
    o = O.Oracle(p, pos=pos, n=n)
    osamples, oedges = [], []
    for b in range(blocks):
        tg, _ = g.cycle_traced(steps, x0, n_c)
        to, _ = o.cycle(steps, x0, n_c, trace=True)
        if not np.array_equal(tg["accepted"], to["accepted"]):
            return g, o, None                   # a near tie: the chains part (checked elsewhere)
        g.structure_sample()
        smp, edges = oracle_samples(p, o, spec)
        osamples.append(smp)
        oedges.append(edges)
    out = ST.concat(osamples)
    out["edges"] = ST.concat_edges(oedges)
    return g, o, out


def compare_reweight(g, p, osmp, spec, kq, mq, n_lo, n_hi):
    """Both sides solve the MBAR equations to convergence (the GPU by the
    accelerated self-consistent iteration, the oracle by the plain one).

    The sampled energies differ by the binary32 pair terms of the GPU path, so
    every reduced potential differs by at most d = max beta |E_gpu - E_oracle|;
    then each D_n and f_s moves by at most 2 d, each weight by a factor within
    exp(+-4 d), and p, rho and g_xy (ratios of positive sums) by at most 8 d
    relative, plus 2e-5 for the binary32 sums over chunks of 256 samples."""
    rg = g.structure_reweight(kq, mq, n_lo, n_hi, tol=1e-11, max_iter=100000)
    ro = ST.reweight(p, osmp, spec, kq, mq, n_lo, n_hi, tol=1e-11)
    e_gpu = g.structure_get()["E"]
    beta = max(1.0 / np.min(p.kT), 1.0 / np.min(kq))
    d = beta * float(np.max(np.abs(e_gpu - osmp["E"])))
    print("max |beta dE| over the samples: %.3g" % d)
    np.testing.assert_allclose(rg["f"], ro["f"], rtol=0, atol=2 * d + 1e-9)
    rel = 8 * d + 2e-5                   # + the binary32 chunk sums of the accumulation
    # phases of probability below 1e-250 are carried by subnormal weights,
    # whose precision is lost on both sides: only their smallness is compared
    big = ro["p"] > 1e-250
    assert np.all(rg["p"][~big] < 1e-240)
    np.testing.assert_allclose(rg["p"][big], ro["p"][big], rtol=rel, atol=0)
    for k in ("rho", "gxy"):
        scale = np.max(np.abs(ro[k][big])) + 1e-300
        np.testing.assert_allclose(rg[k][big], ro[k][big], rtol=rel, atol=1e-12 * scale)
    return rg, ro


def test_paper_run_in_lockstep_samples():
    """160 replicas of the LJ A18 system, x0 = 0.99, a sample every 100 steps:
    the samples equal the oracle's; the GPU's averages over them keep their
    invariants (p sums to 1 over the phases; the 400 slabs of 0.12 A cover the
    48 A zone, so rho integrates to N_B)."""
    p = W.lj_a18_slab(nmax=128, seed=5)
    rng = np.random.default_rng(7)
    pos, n = W.lj_a18_initial(p, rng.integers(0, 100, p.S), seed=8)
    spec = spec_of(p)
    g, o, osmp = run_lockstep_with_samples(p, pos, n, blocks=4, steps=100, x0=0.99, n_c=10, spec=spec)
    if osmp is None:
        pytest.skip("the chains parted at a near tie before the samples were complete")
    assert_same_samples(g.structure_get(), osmp, osmp["edges"])
    kq = p.kT[[0, 5, 9]]
    mq = p.mu[[8, 12, 15]]
    rg = g.structure_reweight(kq, mq, 0, p.nmax, tol=1e-10, max_iter=100000)
    np.testing.assert_allclose(rg["p"].sum(axis=1), 1.0, rtol=1e-9)
    ok = rg["p"] > 1e-12
    A = p.Lx * p.Ly
    integral = rg["rho"].sum(axis=2) * A * float(np.float32(spec["dz"]))
    nb = np.broadcast_to(np.arange(p.nmax + 1), integral.shape)
    # a particle on the top wall is past slab 399; 2e-5: the binary32 chunk sums
    assert np.all(integral[ok] <= nb[ok] * (1 + 2e-5))
    np.testing.assert_allclose(integral[ok], nb[ok], rtol=1e-3)


def test_lj_slab_narrow_grid_reweighted():
    """A 4 x 4 block of the LJ A18 grid (400-550 K, -1.6..-1.3 eV), whose
    neighbouring states overlap: MBAR per phase at sampled and unsampled
    states against the oracle's."""
    base = W.lj_a18_slab(nmax=128, seed=9)
    p = base.replace(kT=W.K_B_EV * np.array([400.0, 450.0, 500.0, 550.0]), mu=np.array([-1.6, -1.5, -1.4, -1.3]))
    rng = np.random.default_rng(2)
    pos, n = W.lj_a18_initial(p, rng.integers(60, 100, p.S), seed=3)
    spec = spec_of(p)
    g, o, osmp = run_lockstep_with_samples(p, pos, n, blocks=16, steps=50, x0=0.9, n_c=10, spec=spec)
    if osmp is None:
        pytest.skip("the chains parted at a near tie before the samples were complete")
    assert_same_samples(g.structure_get(), osmp, osmp["edges"])
    kB = W.K_B_EV
    kq = np.array([p.kT[1], p.kT[2], kB * 475.0, kB * 520.0])
    mq = np.array([p.mu[1], p.mu[2], -1.45, -1.38])
    compare_reweight(g, p, osmp, spec, kq, mq, int(osmp["N"].min()), int(osmp["N"].max()))


def test_small_grid_lockstep_reweight_at_unsampled_states():
    p = W.fcc100_small(seed=11)
    pos, n = W.initial_walkers(p, 12, seed=3)
    spec = {"n_z": 75, "dz": 0.12, "layers": [(p.z_lo, p.z_lo + 1.0), (p.z_lo + 1.0, p.z_lo + 2.2)],
            "n_r": 30, "dr": 0.1}
    g, o, osmp = run_lockstep_with_samples(p, pos, n, blocks=12, steps=20, x0=0.9, n_c=10, spec=spec)
    if osmp is None:
        pytest.skip("the chains parted at a near tie before the samples were complete")
    assert_same_samples(g.structure_get(), osmp, osmp["edges"])
    kq = np.array([0.7, 1.2, p.kT[2]])
    mq = np.array([-5.0, -2.5, p.mu[1]])
    rg, _ = compare_reweight(g, p, osmp, spec, kq, mq, 0, p.nmax)
    # the 75 slabs cover the gas region: rho integrates to N_B in every phase
    A = p.Lx * p.Ly
    ok = rg["p"] > 1e-12
    integral = rg["rho"].sum(axis=2) * A * float(np.float32(spec["dz"]))
    nb = np.broadcast_to(np.arange(p.nmax + 1), integral.shape)
    np.testing.assert_allclose(integral[ok], nb[ok], rtol=2e-5)      # the binary32 chunk sums


def test_store_limits_and_arguments():
    p = W.fcc100_small(L=2, M=2, seed=12)
    pos, n = W.initial_walkers(p, 6, seed=1)
    g = Regc(p)
    g.set_walkers(pos, n)
    with pytest.raises(Exception):
        g.structure_sample()                                   # no store yet
    for bad in ((0, 0.1, [], 10, 0.1, 8), (10, 0.0, [], 10, 0.1, 8), (10, 0.1, [], 10, 0.5, 8),
                (10, 0.1, [(2.0, 1.0)], 10, 0.1, 8), (10, 0.1, [], 10, 0.1, 0)):
        with pytest.raises(Exception):
            g.structure_init(*bad)
    g.structure_init(20, 0.5, [(p.z_lo, p.z_lo + 1.0)], 20, 0.1, 2 * p.S)
    with pytest.raises(Exception):
        g.structure_reweight([1.0], [-3.0], 0, 5)             # no samples yet
    g.structure_sample()
    g.structure_sample()
    with pytest.raises(Exception):
        g.structure_sample()                                   # full: nothing appended
    assert g.structure_count() == 2 * p.S
    r = g.structure_reweight([1.0], [-3.0], 0, p.nmax)
    assert abs(r["p"].sum() - 1.0) < 1e-9
    g.structure_reset()
    assert g.structure_count() == 0
    g.structure_sample()
    assert g.structure_count() == p.S


def test_aiat_matches_oracle():
    """aiAT@REGC (Eq. aiTherm) over the lock-step samples of the LJ A18
    narrow grid: the lowest energy per composition equals the oracle's within
    the energy tolerance, the stable composition agrees wherever the two
    lowest dG are further apart than that tolerance, and the configuration
    kept for a composition has that composition and that energy."""
    base = W.lj_a18_slab(nmax=128, seed=13)
    p = base.replace(kT=W.K_B_EV * np.array([400.0, 450.0, 500.0, 550.0]), mu=np.array([-1.6, -1.5, -1.4, -1.3]))
    rng = np.random.default_rng(5)
    pos, n = W.lj_a18_initial(p, rng.integers(40, 100, p.S), seed=6)
    spec = spec_of(p)
    g, o, osmp = run_lockstep_with_samples(p, pos, n, blocks=10, steps=40, x0=0.9, n_c=10, spec=spec)
    if osmp is None:
        pytest.skip("the chains parted at a near tie before the samples were complete")
    mu_q = np.linspace(-2.4, -0.9, 31)
    e_g, dG_g, ph_g = g.aiat(mu_q)
    e_o, first = AI.lowest_energy(osmp["N"], osmp["E"], p.nmax)
    dG_o, ph_o = AI.formation_free_energy(e_o, mu_q)
    assert np.array_equal(np.isnan(e_g), np.isnan(e_o))
    seen = ~np.isnan(e_o)
    tol = 1e-4 * np.maximum(1.0, np.abs(e_o[seen]))
    assert np.all(np.abs(e_g[seen] - e_o[seen]) <= tol)
    for q in range(len(mu_q)):
        srt = np.sort(dG_o[q][np.isfinite(dG_o[q])])
        if len(srt) > 1 and srt[1] - srt[0] > 2e-4 * max(1.0, abs(srt[0])):
            assert ph_g[q] == ph_o[q], (mu_q[q], ph_g[q], ph_o[q])
    # the kept configurations: composition and energy
    for nb in np.nonzero(seen)[0][:: max(1, int(seen.sum()) // 6)]:
        xyz = g.aiat_config(int(nb))
        assert len(xyz) == nb
        h = Regc(p)
        one = np.zeros((p.S, p.nmax, 3), np.float32)
        one[0, :nb] = xyz
        cnt = np.zeros(p.S, np.int32)
        cnt[0] = nb
        h.set_walkers(one, cnt)
        assert h.get_walkers()[2][0] == e_g[nb]                # the exact fixed-point energy
        h.close()
    g.structure_reset()
    e_r, _, _ = g.aiat([0.0])
    assert np.all(np.isnan(e_r))
    with pytest.raises(Exception):
        g.aiat_config(int(np.nonzero(seen)[0][0]))


def test_structure_edge_cases():
    """Walkers at N = 0 and at N = Nmax, a periodic box (the slab counts span
    the whole cell), no layers at all, a single distance bin; every count
    equal to the oracle's."""
    p = W.ideal_gas(W.fcc100_small(L=2, M=2, nmax=24, seed=15)).replace(
        periodic_z=1, z_lo=0.0, z_hi=10.0, Lz=10.0, surf_xyz=np.zeros((0, 3)), surf_type=np.zeros(0, np.int32))
    pos, n = W.initial_walkers(p, [0, 24, 1, 13], seed=9, min_dist=0.5)
    g = Regc(p)
    g.set_walkers(pos, n)
    o = O.Oracle(p, pos=pos, n=n)
    for spec in ({"n_z": 84, "dz": 0.12, "layers": [], "n_r": 1, "dr": 3.0},
                 {"n_z": 1, "dz": 10.0, "layers": [(0.0, 10.0), (2.0, 2.5), (9.5, 10.0), (0.0, 0.1)], "n_r": 31,
                  "dr": 0.1}):
        init_store(g, spec, p.S)
        g.structure_sample()
        gs = g.structure_get()
        os_, edges = oracle_samples(p, o, spec)
        assert_same_samples(gs, os_, edges)
        assert gs["rho"].sum() == n.sum() if spec["n_z"] == 84 else True
    # empty store: aiAT has no composition; reweighting is refused
    g.structure_reset()
    e_min, dG, ph = g.aiat([-1.0, 1.0])
    assert np.all(np.isnan(e_min)) and np.all(np.isinf(dG)) and list(ph) == [-1, -1]
    with pytest.raises(Exception):
        g.structure_reweight([1.0], [-3.0], 0, 3)
