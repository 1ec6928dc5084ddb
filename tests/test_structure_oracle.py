"""Pins of the structure oracle (Sec. III.A "Structural properties": the axial
distribution rho(z) in slabs of 0.12 A and the lateral RDF g_xy(r) of an
adsorbate layer; Sec. II.B, Eq. avegr: their MBAR averages per phase).

* Closed forms of one configuration: the 36 hollow sites of the top A layer of
  the LJ A18 system form a honeycomb net whose pair shells (a/sqrt(3): 3
  neighbours, a: 6, 2a/sqrt(3): 3) fix the pair counts; particles at known
  heights fix the slab counts.
* Uniformly placed points have g_xy = 1 on average in every shell (the
  normalisation); a doubled pair count (planted) is caught.
* One sampled state: the MBAR average of each phase is the plain average of
  its samples.
* The ideal gas sampled by the oracle's REGC run, reweighted to a state that
  was not sampled: p(N) is the truncated Poisson law there, rho(z) within a
  phase is flat at N/(A H), and rho integrates to N exactly; leaving the
  3 N ln Lambda term out of the query (planted) is caught, and so is a slab
  index off by one.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from oracle import structure as ST
from test_oracle_pins import ideal_lambda, trunc_poisson


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def hollow_sites(p):
    """The 36 hollow sites (both kinds) of the B-stacked top layer of the LJ
    A18 cell: two triangular nets of spacing a, shifted by (0, 0) and
    (a, 2h/3) from the bottom layer's net."""
    a = 11.489 / 3.0
    h = a * math.sqrt(3.0) / 2.0
    pts = []
    for sx, sy in ((0.0, 0.0), (a, 2.0 * h / 3.0)):
        for j in range(6):
            for i in range(3):
                pts.append(((i * a + (0.5 * a if j % 2 else 0.0) + sx) % p.Lx, (j * h + sy) % p.Ly))
    xy = W.f32(np.array(pts))
    # a coordinate that rounds up onto the period is the image at 0
    xy[:, 0] = np.where(xy[:, 0] >= p.Lx, 0.0, xy[:, 0])
    xy[:, 1] = np.where(xy[:, 1] >= p.Ly, 0.0, xy[:, 1])
    return xy, a


def test_honeycomb_pair_shells_and_one_slab():
    p = W.lj_a18_slab(L=1, M=1, nmax=64)
    xy, a = hollow_sites(p)
    pos = np.zeros((p.nmax, 3))
    pos[:36, :2] = xy
    pos[:36, 2] = p.z_lo + 0.05
    pos = W.f32(pos)
    spec = {"n_z": 400, "dz": 0.12, "layers": [(p.z_lo, p.z_lo + 1.0), (p.z_lo + 1.0, p.z_lo + 2.0)],
            "n_r": 57, "dr": 0.1}
    rho, pairs, pop = ST.sample_counts(p, pos, 36, spec)
    assert rho[0] == 36 and rho.sum() == 36
    assert list(pop) == [36, 0]
    want = np.zeros(57, np.int64)
    for d, z in ((a / math.sqrt(3.0), 3), (a, 6), (2.0 * a / math.sqrt(3.0), 3)):
        want[int(d / 0.1)] += 36 * z // 2
    assert np.array_equal(pairs[0], want), (np.nonzero(pairs[0]), np.nonzero(want))
    assert pairs[1].sum() == 0


def test_slab_counts_at_known_heights():
    p = W.lj_a18_slab(L=1, M=1, nmax=16)
    ks = [0, 3, 3, 17, 399]
    pos = np.zeros((p.nmax, 3))
    pos[:5, 0] = 1.0
    pos[:5, 1] = 2.0
    pos[:5, 2] = [p.z_lo + (k + 0.5) * 0.12 for k in ks]
    pos[5] = [3.0, 3.0, p.z_hi]                      # on the top wall: above slab 399
    pos = W.f32(pos)
    spec = {"n_z": 400, "dz": 0.12, "layers": [], "n_r": 10, "dr": 0.5}
    rho, _, _ = ST.sample_counts(p, pos, 6, spec)
    assert np.array_equal(np.nonzero(rho)[0], [0, 3, 17, 399]) and rho[3] == 2 and rho.sum() == 5
    rho_bad, _, _ = ST.sample_counts(p, pos, 6, spec, mutation=1)
    assert not np.array_equal(rho_bad, rho)


def uniform_layer_g(mutation=0, n_conf=300, m=30, seed=3):
    p = W.lj_a18_slab(L=1, M=1, nmax=64)
    rng = np.random.default_rng(seed)
    spec = {"n_z": 10, "dz": 1.0, "layers": [(p.z_lo, p.z_lo + 1.0)], "n_r": 57, "dr": 0.1}
    A = p.Lx * p.Ly
    shell = math.pi * 0.01 * ((np.arange(57) + 1.0) ** 2 - np.arange(57) ** 2)
    gs = []
    for c in range(n_conf):
        pos = np.zeros((p.nmax, 3))
        pos[:m] = np.stack([rng.uniform(0, p.Lx, m), rng.uniform(0, p.Ly, m), p.z_lo + rng.uniform(0, 1, m)], 1)
        pos = W.f32(pos)
        pos[:m, 0] = np.where(pos[:m, 0] >= p.Lx, 0.0, pos[:m, 0])
        pos[:m, 1] = np.where(pos[:m, 1] >= p.Ly, 0.0, pos[:m, 1])
        _, pairs, pop = ST.sample_counts(p, pos, m, spec, mutation=mutation)
        gs.append(2.0 * A * pairs[0] / (pop[0] * (pop[0] - 1.0)) / shell)
    gs = np.array(gs)[:, 10:]                       # shells with enough pairs for a mean
    return gs.mean(), gs.mean(axis=1).std(ddof=1) / math.sqrt(n_conf)


def test_uniform_points_have_unit_rdf():
    mean, se = uniform_layer_g()
    assert abs(mean - 1.0) < 4.5 * se, (mean, se)
    mean2, se2 = uniform_layer_g(mutation=2, n_conf=40)
    assert abs(mean2 - 1.0) > 10 * se2


def test_one_state_average_is_the_plain_average():
    p = W.fcc100_small(L=1, M=1, nmax=24, seed=2)
    spec = {"n_z": 60, "dz": 0.12, "layers": [(p.z_lo, p.z_lo + 1.5)], "n_r": 20, "dr": 0.15}
    rng = np.random.default_rng(1)
    samples = []
    for c in range(40):
        pos, n = W.initial_walkers(p, rng.integers(3, 8), seed=c)
        o = O.Oracle(p, pos=pos, n=n)
        samples.append(ST.structure_of_walkers(p, o.pos, o.n, o.state_of_walker, o.energy, spec))
    smp = ST.concat(samples)
    out = ST.reweight(p, smp, spec, p.kT[:1], p.mu[:1], 3, 7)
    A = p.Lx * p.Ly
    for i, nb in enumerate(range(3, 8)):
        sel = smp["N"] == nb
        assert out["p"][0, i] == pytest.approx(sel.mean(), rel=1e-12)
        if sel.any():
            dz = float(np.float32(0.12))                # widths are binary32 values
            np.testing.assert_allclose(out["rho"][0, i], smp["rho"][sel].mean(axis=0) / (A * dz), rtol=1e-11)


def ideal_gas_run(seed=0, blocks=300):
    p = W.ideal_gas(W.fcc100_small(seed=seed))
    spec = {"n_z": 75, "dz": 0.12, "layers": [(p.z_lo, p.z_lo + 2.0)], "n_r": 20, "dr": 0.15}
    o = O.Oracle(p)
    o.run(50, exchange_every=5, hist=False)
    samples = []
    for b in range(blocks):
        o.run(5, exchange_every=5, hist=False)
        samples.append(ST.structure_of_walkers(p, o.pos, o.n, o.state_of_walker, o.energy, spec))
    return p, spec, ST.concat(samples)


@pytest.fixture(scope="module")
def ideal():
    return ideal_gas_run()


QUERIES = [(1.3, -3.0), (0.65, -4.0)]      # off the sampled grid, inside its range


def ideal_pin(ideal, mutation=0):
    """Largest |z| of <N> at unsampled states against the truncated Poisson
    mean, and the reweighted averages of the first query."""
    p, spec, smp = ideal
    kq = np.array([q[0] for q in QUERIES])
    mq = np.array([q[1] for q in QUERIES])
    out = ST.reweight(p, smp, spec, kq, mq, 0, p.nmax, mutation=mutation)
    nv = np.arange(p.nmax + 1)
    n_eff = len(smp["N"]) / p.S / 3.0          # samples per state, thinned for their correlation
    worst = 0.0
    for i in range(len(QUERIES)):
        q = p.replace(kT=kq[i:i + 1], mu=mq[i:i + 1])
        pr = trunc_poisson(ideal_lambda(q, 0), p.nmax)
        mean, sd = pr @ nv, math.sqrt(pr @ nv ** 2 - (pr @ nv) ** 2)
        worst = max(worst, abs(out["p"][i] @ nv - mean) / (sd / math.sqrt(n_eff)))
    return worst, out


def test_ideal_gas_reweighted_to_an_unsampled_state(ideal):
    z, out = ideal_pin(ideal)
    assert z < 4.5, z
    p, spec, smp = ideal
    A, H = p.Lx * p.Ly, p.z_hi - p.z_lo
    nb = np.arange(p.nmax + 1)
    ok = out["p"][0] > 1e-3
    # the 75 slabs of 0.12 cover the whole region (H = 8.895): rho integrates
    # to N in every phase
    integral = out["rho"][0].sum(axis=1) * A * float(np.float32(spec["dz"]))
    np.testing.assert_allclose(integral[ok], nb[ok], rtol=1e-12)
    # and is flat at N / (A H) over the 74 slabs inside the region
    flat = nb[ok] / (A * H)
    mean = out["rho"][0][ok][:, :74].mean(axis=1)
    np.testing.assert_allclose(mean, flat, rtol=0.1)


def test_ideal_gas_planted_lambda_mistake_is_detected(ideal):
    z, _ = ideal_pin(ideal, mutation=4)
    assert z > 6.0, z
