"""Pins of the oracle's second grand-canonical species (more than one
reactive gas, the outlook of Sec. IV): species B and C, each inserted and
removed by the rules of Sec. II.A.1 with its own chemical potential and
thermal wavelength, on a (T, mu_B, mu_C) grid whose neighbours swap by the
rule of Eq. Pacc extended to both species.

* Every acceptance ratio, including the swap, against the ratio of the
  two-species grand-canonical densities (Eq. Ngrand with a product over
  species: V^N / (Lambda_B^{3 N_B} Lambda_C^{3 N_C} N_B! N_C!)
  exp(-beta (E - mu_B N_B - mu_C N_C))).
* The ideal gas (every eps = 0) with replica exchange along all five grid
  directions: (N_B, N_C) follows the product of two Poisson laws truncated to
  N_B + N_C <= Nmax, so <N_B> and <N_C> are known at every state.
* A small box with Nmax = 2 against brute-force integrals of the partition
  function: one and two particles of either species, and the B-C pair.
* The running energy against a from-scratch recompute.
* Planted mistakes (C inserted with B's mu and Lambda; the swap without the
  mu_C term) are caught.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from test_oracle_pins import lj_np


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def log_density2(p, state, nb, nc, energy):
    kT, mu, mu2 = (x[state] for x in p.state_params())
    lb = p.lambda0 / math.sqrt(kT)
    lc = p.lambda0_2 / math.sqrt(kT)
    return ((mu * nb + mu2 * nc - energy) / kT + (nb + nc) * math.log(p.volume)
            - 3 * nb * math.log(lb) - 3 * nc * math.log(lc) - math.lgamma(nb + 1) - math.lgamma(nc + 1))


def pin_acceptance2(mutation=0):
    p = W.two_gas_small()
    orc = O.Oracle(p, mutation=mutation)
    rng = np.random.default_rng(4)
    worst = 0.0
    for _ in range(300):
        s = int(rng.integers(p.S))
        nb, nc = (int(x) for x in rng.integers(1, 12, 2))
        e0, de = rng.normal() * 5, rng.normal() * 3
        for sp, (db, dc) in ((0, (1, 0)), (1, (0, 1))):
            ins = log_density2(p, s, nb + db, nc + dc, e0 + de) - log_density2(p, s, nb, nc, e0)
            rem = log_density2(p, s, nb - db, nc - dc, e0 + de) - log_density2(p, s, nb, nc, e0)
            n_c = nc if sp else nb
            worst = max(worst, abs(orc.log_alpha2(1, sp, s, n_c, de) - ins),
                        abs(orc.log_alpha2(2, sp, s, n_c, de) - rem))
        sa, sb = (int(x) for x in rng.choice(p.S, 2, replace=False))
        na_b, na_c, nb_b, nb_c = (int(x) for x in rng.integers(0, 16, 4))
        ea, eb = rng.normal(size=2) * 10
        swap = (log_density2(p, sa, nb_b, nb_c, eb) + log_density2(p, sb, na_b, na_c, ea)
                - log_density2(p, sa, na_b, na_c, ea) - log_density2(p, sb, nb_b, nb_c, eb))
        worst = max(worst, abs(orc.exchange_log_alpha2(sa, sb, na_b, na_c, nb_b, nb_c, ea, eb) - swap))
    return worst


def test_acceptance_ratios_are_density_ratios():
    assert pin_acceptance2() < 1e-9


def trunc_joint_means(lb, lc, nmax):
    """<N_B>, <N_C> of P(a, b) ~ lb^a / a! lc^b / b!, a + b <= nmax."""
    a = np.arange(nmax + 1)
    la = a * math.log(lb) - np.array([math.lgamma(k + 1) for k in a])
    lcv = a * math.log(lc) - np.array([math.lgamma(k + 1) for k in a])
    lp = la[:, None] + lcv[None, :]
    lp[a[:, None] + a[None, :] > nmax] = -np.inf
    w = np.exp(lp - lp.max())
    w /= w.sum()
    return float(w.sum(axis=1) @ a), float(w.sum(axis=0) @ a), w


def pin_ideal2(mutation=0, n_batches=12, sweeps=300):
    """Largest |z| of per-state <N_B>, <N_C> against the truncated product of
    Poisson laws, with a swap attempt after every sweep (few particle moves
    between swaps, so that a wrong swap rule shows)."""
    p = W.ideal_gas(W.two_gas_small(L=2, M=3, K=3, nmax=16)).replace(
        kT=np.array([0.9, 1.1]), mu=np.array([-4.6, -4.3, -4.0]), mu2=np.array([-4.8, -4.4, -4.0]),
        moves_per_sweep=4, p_disp=0.0)
    orc = O.Oracle(p, mutation=mutation)
    kT, mu, mu2 = p.state_params()
    exp_b, exp_c = np.zeros(p.S), np.zeros(p.S)
    for s in range(p.S):
        lb = p.volume * math.exp(mu[s] / kT[s]) / (p.lambda0 / math.sqrt(kT[s])) ** 3
        lc = p.volume * math.exp(mu2[s] / kT[s]) / (p.lambda0_2 / math.sqrt(kT[s])) ** 3
        exp_b[s], exp_c[s], _ = trunc_joint_means(lb, lc, p.nmax)
    orc.run(200, exchange_every=1, hist=False)
    nbm, ncm = np.zeros((n_batches, p.S)), np.zeros((n_batches, p.S))
    nv = np.arange(p.nmax + 1)
    for b in range(n_batches):
        h0, h20 = orc.hN.copy(), orc.hN2.copy()
        orc.run(sweeps, exchange_every=1)
        dh, dh2 = orc.hN - h0, orc.hN2 - h20
        nbm[b] = (dh @ nv) / np.maximum(dh.sum(axis=1), 1)
        ncm[b] = (dh2 @ nv) / np.maximum(dh2.sum(axis=1), 1)
    assert orc.ex_counts[:, 4, 1].sum() > 0          # swaps along mu_C happened
    z = []
    for m, ex in ((nbm, exp_b), (ncm, exp_c)):
        se = np.maximum(m.std(axis=0, ddof=1) / math.sqrt(n_batches), 1e-3)
        z.append(np.abs(m.mean(axis=0) - ex) / se)
    return float(np.max(z)), exp_b, exp_c


def test_ideal_gas_two_species_with_exchange():
    z, exp_b, exp_c = pin_ideal2()
    # the cap N_B + N_C <= 16 matters at some states
    assert np.max(exp_b + exp_c) > 12
    assert z < 4.5


def test_planted_species_and_swap_mistakes_are_caught():
    assert pin_acceptance2(mutation=32768) > 0.1
    assert pin_acceptance2(mutation=65536) > 0.1
    assert pin_ideal2(mutation=32768, n_batches=8, sweeps=200)[0] > 6
    assert pin_ideal2(mutation=65536, n_batches=8, sweeps=200)[0] > 6


def small_box2():
    """The small box of the single-species pin (5.2 x 5.2, 4 surface atoms,
    gas 1.0 <= z <= 3.0, rc 2.5, Nmax 2) with both species on a 2 x 2 x 2 grid."""
    surf = W.f32(np.array([[0.0, 0.0, 0.0], [2.6, 0.0, 0.0], [0.0, 2.6, 0.0], [2.6, 2.6, 0.0]]))
    eps = np.zeros((4, 4))
    sig = np.ones((4, 4))
    eps[0, 0] = 1.0
    eps[0, 1] = eps[1, 0] = 1.5
    eps[2, 2], sig[2, 2] = 0.7, 0.9
    eps[0, 2] = eps[2, 0] = 1.1
    sig[0, 2] = sig[2, 0] = 0.95
    eps[1, 2] = eps[2, 1] = 1.0
    sig[1, 2] = sig[2, 1] = 1.05
    return W.Problem(
        n_types=3, eps=eps, sigma=sig, rc=2.5, Lx=5.2, Ly=5.2, Lz=3.0, periodic_z=0,
        z_lo=1.0, z_hi=3.0, surf_xyz=surf, surf_type=np.ones(4, np.int32),
        kT=np.array([0.9, 1.3]), mu=np.array([-5.5, -4.0]), lambda0=1.0, nmax=2,
        moves_per_sweep=20, max_disp=0.4, p_disp=1.0 / 3.0, seed=7,
        e_lo=W.centred_e_lo(-40.0, 0.05), e_bin=0.05, n_e_bins=1600, name="small_box2",
        gc2_type=2, mu2=np.array([-5.0, -3.8]), lambda0_2=0.8)


def e_surf2(p, pts, c):
    e = np.zeros(len(pts))
    for a in p.surf_xyz:
        d = pts - a
        d[:, 0] -= p.Lx * np.round(d[:, 0] / p.Lx)
        d[:, 1] -= p.Ly * np.round(d[:, 1] / p.Ly)
        e += lj_np(np.sum(d * d, axis=1), p.eps[c, 1], p.sigma[c, 1], p.rc)
    return e


def brute_force2(p, n_grid=(96, 96, 60), n_mc=2_000_000, seed=13):
    """Per temperature and species pair: Z and <E | composition> of the
    compositions (1, 0), (0, 1), (2, 0), (1, 1), (0, 2) -- one-particle
    integrals by the midpoint rule, the pair parts by Monte Carlo over the
    cutoff ball (as the single-species pin)."""
    nx, ny, nz = n_grid
    hx, hy, hz = p.Lx / nx, p.Ly / ny, (p.z_hi - p.z_lo) / nz
    X, Y, Z = np.meshgrid((np.arange(nx) + 0.5) * hx, (np.arange(ny) + 0.5) * hy,
                          p.z_lo + (np.arange(nz) + 0.5) * hz, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    dv = hx * hy * hz
    es = {c: e_surf2(p, grid, c) for c in (0, 2)}
    rng = np.random.default_rng(seed)
    V = p.volume
    vball = 4.0 / 3.0 * math.pi * p.rc ** 3
    r1 = np.stack([rng.uniform(0, p.Lx, n_mc), rng.uniform(0, p.Ly, n_mc), rng.uniform(p.z_lo, p.z_hi, n_mc)], 1)
    d = rng.normal(size=(n_mc, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    d *= (p.rc * rng.uniform(0, 1, n_mc) ** (1.0 / 3.0))[:, None]
    r2 = r1 + d
    inside = (r2[:, 2] >= p.z_lo) & (r2[:, 2] <= p.z_hi)
    r2[:, 0] %= p.Lx
    r2[:, 1] %= p.Ly
    d2 = np.sum(d * d, axis=1)
    out = {}
    for kT in p.kT:
        b = 1.0 / kT
        z1, i1 = {}, {}
        for c in (0, 2):
            g = np.exp(-b * es[c])
            z1[c] = g.sum() * dv
            i1[c] = (es[c] * g).sum() * dv
        pair = {}
        for (c1, c2) in ((0, 0), (0, 2), (2, 2)):
            e1, e2 = e_surf2(p, r1, c1), e_surf2(p, r2, c2)
            phi = lj_np(d2, p.eps[c1, c2], p.sigma[c1, c2], p.rc)
            gg = np.exp(-b * (e1 + e2)) * inside
            mayer = V * vball * np.mean(gg * (np.exp(-b * phi) - 1.0))
            emayer = V * vball * np.mean(gg * (np.exp(-b * phi) * (e1 + e2 + phi) - (e1 + e2)))
            zz = z1[c1] * z1[c2] + mayer
            ee = (z1[c1] * i1[c2] + z1[c2] * i1[c1] + emayer) / zz
            pair[(c1, c2)] = (zz, ee)
        out[float(kT)] = (z1, i1, pair)
    return out


def small_box2_expected(p, bf):
    """Exact <N_B>, <N_C>, <E> per state: compositions (a, b) with a + b <= 2,
    weight z_B^a z_C^b Z_(a,b) / (a! b!), z_c = exp(beta mu_c) / Lambda_c^3."""
    kT, mu, mu2 = p.state_params()
    out = np.zeros((p.S, 3))
    for s in range(p.S):
        z1, i1, pair = bf[float(kT[s])]
        zb = math.exp(mu[s] / kT[s]) / (p.lambda0 / math.sqrt(kT[s])) ** 3
        zc = math.exp(mu2[s] / kT[s]) / (p.lambda0_2 / math.sqrt(kT[s])) ** 3
        comps = [((0, 0), 1.0, 0.0), ((1, 0), zb * z1[0], i1[0] / z1[0]), ((0, 1), zc * z1[2], i1[2] / z1[2]),
                 ((2, 0), zb * zb * pair[(0, 0)][0] / 2, pair[(0, 0)][1]),
                 ((1, 1), zb * zc * pair[(0, 2)][0], pair[(0, 2)][1]),
                 ((0, 2), zc * zc * pair[(2, 2)][0] / 2, pair[(2, 2)][1])]
        w = np.array([c[1] for c in comps])
        w /= w.sum()
        out[s, 0] = sum(wi * c[0][0] for wi, c in zip(w, comps))
        out[s, 1] = sum(wi * c[0][1] for wi, c in zip(w, comps))
        out[s, 2] = sum(wi * c[2] for wi, c in zip(w, comps))
    return out


@pytest.mark.slow
def test_small_box_two_species_brute_force():
    p = small_box2()
    exp = small_box2_expected(p, brute_force2(p))
    runs = []
    for r in range(8):
        o = O.Oracle(p.replace(seed=300 + r))
        o.run(500, exchange_every=10, hist=False)
        o.run(8000, exchange_every=10)
        runs.append(np.stack([o.moments[:, 0] / o.omega, o.moments2[:, 0] / o.omega,
                              o.moments[:, 2] / o.omega], axis=1))
    runs = np.array(runs)
    m, se = runs.mean(0), runs.std(0, ddof=1) / math.sqrt(len(runs))
    z = np.abs(m - exp) / np.maximum(se, 1e-4)
    assert z.max() < 4.5, (z, m, exp)


def test_running_energy_matches_recompute_two_species():
    p = W.two_gas_small()
    pos, n, nb = W.two_gas_initial(p, 10, 8, seed=3)
    o = O.Oracle(p, pos=pos, n=n, nb=nb)
    o.run(150, exchange_every=10, hist=False)
    assert np.all(o.nb <= o.n) and (o.nb > 0).any() and (o.n - o.nb > 0).any()
    err = max(abs(o.energy[w] - o.total_energy(w)) for w in range(p.S))
    assert err < 1e-8
