"""Pins of the oracle's second mobile species (the cluster of the cluster-in-gas
workload; not in the paper).

* Pair energies of each species pair against the closed-form 12-6 terms.
* An invisible cluster (eps_AB = 0) leaves the grand-canonical species an ideal
  gas: N_B follows the truncated Poisson distribution of Eq. Ngrand, with the
  cluster displacing among the moves; a planted mistake that uses the total N
  in the insertion/removal ratios is detected.
* One cluster atom in a periodic box with up to two B particles: <N_B> and <E>
  against brute-force configuration integrals (by translation invariance the
  atom can be held at the centre).
* The running energy equals the from-scratch energy after sweeps of the
  cfg-5 system, and cluster atoms are never removed or renumbered.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from test_oracle_pins import batch_means, lj_np, trunc_poisson, zscores


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def test_species_pair_energies_closed_form():
    p = W.cluster_in_gas(L=1, M=1, nmax_b=4)
    pos = np.zeros((1, p.nmax, 3))
    pos[0, :4] = [[5.0, 5.0, 5.0], [6.25, 5.0, 5.0], [5.0, 9.0, 5.0], [5.0, 5.0, 9.0]]
    pos[0, 4] = [7.0, 5.0, 5.0]            # a B particle
    o = O.Oracle(p, pos=pos, n=np.array([5], np.int32))
    eps, sig, rc2 = p.eps, p.sigma, p.rc ** 2

    def phi(a, b, ta, tb):                  # closed-form truncated 12-6 term of two points
        r2 = float(np.sum((np.asarray(a) - np.asarray(b)) ** 2))
        if r2 >= rc2:
            return 0.0
        s6 = (sig[ta, tb] ** 2 / r2) ** 3
        return 4.0 * eps[ta, tb] * (s6 * s6 - s6)

    typ = [1, 1, 1, 1, 0]
    for i in range(5):
        want = sum(phi(pos[0, i], pos[0, j], typ[i], typ[j]) for j in range(5) if j != i)
        got = o.particle_energy(0, pos[0, i], skip=i)[0]
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12), i
    # a new particle (insertion, skip = -1) is of the grand-canonical species
    q = [5.0, 6.5, 5.0]
    want = sum(phi(q, pos[0, j], 0, typ[j]) for j in range(5))
    assert o.particle_energy(0, np.array(q), skip=-1)[0] == pytest.approx(want, rel=1e-12)
    # the pair types are really distinct here: A-A, A-B and B-new all enter
    assert phi(pos[0, 0], pos[0, 1], 1, 1) != 0.0 and phi(pos[0, 1], pos[0, 4], 1, 0) != 0.0
    tot = sum(phi(pos[0, i], pos[0, j], typ[i], typ[j]) for i in range(5) for j in range(i + 1, 5))
    assert o.total_energy(0) == pytest.approx(tot, rel=1e-12)


def invisible_cluster_problem():
    p = W.cluster_in_gas(L=2, M=2, nmax_b=12, box=6.0, seed=5)
    eps = p.eps.copy()
    eps[0, 0] = 0.0
    eps[0, 1] = eps[1, 0] = 0.0
    return p.replace(eps=eps, mu=np.array([-4.5, -3.5]))


def pin_invisible_cluster(mutation=0, n_batches=16, sweeps=400):
    p = invisible_cluster_problem()
    pos, n = W.cluster_initial(p, 0, seed=1)
    o = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    o.run(100, exchange_every=10, hist=False)
    nb, _ = batch_means(o, n_batches, sweeps, exchange_every=10)
    V = p.Lx * p.Ly * p.Lz
    kmax = p.nmax - p.n_cluster
    exp_mean, exp_sd = np.zeros(p.S), np.zeros(p.S)
    k = np.arange(kmax + 1)
    for s in range(p.S):
        kT, mu = p.kT[s // p.M], p.mu[s % p.M]
        lam = V * math.exp(mu / kT) / (p.lambda0 / math.sqrt(kT)) ** 3
        pr = trunc_poisson(lam, kmax)
        exp_mean[s] = pr @ k
        exp_sd[s] = math.sqrt(pr @ k ** 2 - exp_mean[s] ** 2)
    return float(np.max(np.abs(zscores(nb, exp_mean, exp_sd, n_batches * sweeps))))


def test_invisible_cluster_leaves_an_ideal_gas():
    assert pin_invisible_cluster() < 4.5


def test_planted_total_n_mistake_is_detected():
    assert pin_invisible_cluster(mutation=256, n_batches=8, sweeps=200) > 6.0


def one_atom_problem():
    p = W.cluster_in_gas(L=2, M=2, nmax_b=2, box=5.2, seed=9)
    p = p.replace(n_cluster=1, nmax=3, kT=np.array([0.9, 1.3]), mu=np.array([-5.5, -4.0]), max_disp=0.4)
    return p


def brute_force_one_atom(p, n_grid=48, n_mc=1_500_000, seed=13):
    """{kT: (Z1, Z2, E1, E2)} of up to two B particles around one cluster atom
    held at the centre of the periodic box (midpoint rule for Z1, Mayer-part
    Monte Carlo for Z2, as for the small slab box)."""
    L = p.Lx
    c = np.full(3, L / 2.0)
    h = L / n_grid
    g = (np.arange(n_grid) + 0.5) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def e_a(pts):
        d = pts - c
        d -= L * np.round(d / L)
        return lj_np(np.sum(d * d, axis=1), p.eps[0, 1], p.sigma[0, 1], p.rc)

    eg = e_a(grid)
    dv = h ** 3
    rng = np.random.default_rng(seed)
    vball = 4.0 / 3.0 * math.pi * p.rc ** 3
    r1 = rng.uniform(0, L, size=(n_mc, 3))
    d = rng.normal(size=(n_mc, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    d *= (p.rc * rng.uniform(0, 1, n_mc) ** (1.0 / 3.0))[:, None]
    r2 = (r1 + d) % L
    e1, e2 = e_a(r1), e_a(r2)
    phi = lj_np(np.sum(d * d, axis=1), p.eps[0, 0], p.sigma[0, 0], p.rc)
    V = L ** 3
    out = {}
    for kT in p.kT:
        b = 1.0 / kT
        w = np.exp(-b * eg)
        z1 = w.sum() * dv
        i1 = (eg * w).sum() * dv
        gg = np.exp(-b * (e1 + e2))
        mayer = V * vball * np.mean(gg * (np.exp(-b * phi) - 1.0))
        emayer = V * vball * np.mean(gg * (np.exp(-b * phi) * (e1 + e2 + phi) - (e1 + e2)))
        z2 = z1 * z1 + mayer
        out[float(kT)] = (z1, z2, i1 / z1, (2.0 * z1 * i1 + emayer) / z2)
    return out


def test_one_cluster_atom_brute_force():
    p = one_atom_problem()
    bf = brute_force_one_atom(p)
    exp_n, exp_e, sd_n = (np.zeros(p.S) for _ in range(3))
    for s in range(p.S):
        kT, mu = p.kT[s // p.M], p.mu[s % p.M]
        z1, z2, e1, e2 = bf[float(kT)]
        zz = math.exp(mu / kT) / (p.lambda0 / math.sqrt(kT)) ** 3
        w = np.array([1.0, zz * z1, zz * zz * z2 / 2.0])
        w /= w.sum()
        exp_n[s] = w @ np.arange(3)
        sd_n[s] = math.sqrt(w @ np.arange(3) ** 2 - exp_n[s] ** 2)
        exp_e[s] = w[1] * e1 + w[2] * e2
    pos, n = W.cluster_initial(p, 0, seed=2)
    o = O.Oracle(p, pos=pos, n=n)
    o.run(500, exchange_every=10, hist=False)
    nb, eb = batch_means(o, 16, 3000, exchange_every=10)
    zn = zscores(nb, exp_n, sd_n, 16 * 3000)
    ze = zscores(eb, exp_e, np.ones(p.S), 16 * 3000)
    assert max(np.max(np.abs(zn)), np.max(np.abs(ze))) < 4.5, (zn, ze)


def test_cluster_running_energy_and_identity():
    p = W.cluster_in_gas(L=2, M=2, nmax_b=40, seed=4)
    pos, n = W.cluster_initial(p, [5, 20, 30, 40], seed=3)
    o = O.Oracle(p, pos=pos, n=n)
    before = o.pos[:, :4].copy()
    for _ in range(5):
        o.sweeps(20)
        o.exchange()
    assert np.all(o.n >= p.n_cluster)
    for w in range(p.S):
        assert abs(o.energy[w] - o.total_energy(w)) <= 1e-9 * max(1.0, abs(o.energy[w]))
    # cluster atoms stay in slots 0..3 and move only by small displacements
    d = o.pos[:, :4] - before
    d -= p.Lx * np.round(d / p.Lx)
    assert np.all(np.abs(d) <= 100 * 0.2 + 1e-9)
    # histograms count N_B
    assert o.hN[:, p.nmax - p.n_cluster + 1:].sum() == 0
