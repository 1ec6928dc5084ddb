"""Pins of the FP64 oracle against facts that the paper and the mathematics fix.

Each pin checks the oracle against something other than itself:

* Philox4x32-10 against the generator's published known-answer vectors;
* the pair potential against closed-form facts of the LJ 12-6 function
  (zero at sigma, minimum -eps at 2^(1/6) sigma, zero beyond rc);
* the minimum-image particle energy against an explicit sum over periodic images;
* the incremental energy bookkeeping against a full O(N^2) recompute;
* every acceptance ratio against the ratio of the grand-canonical densities of
  Eq. Ngrand (insertion, removal, displacement, and the swap of Eq. Pacc);
* the sampler against the ideal-gas limit (eps = 0: N is Poisson with mean
  V exp(beta mu) / Lambda^3, truncated at Nmax), with and without replica exchange;
* the sampler with interactions against brute-force partition functions of a
  small box with Nmax = 2 (3-D quadrature and a 6-D Mayer-function integral).

``test_pins_detect_planted_mistakes`` turns on the oracle's planted-mistake
switches one at a time and checks that some pin fails for each.
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def trunc_poisson(lam, nmax):
    n = np.arange(nmax + 1)
    logp = n * np.log(lam) - np.array([math.lgamma(k + 1) for k in n])
    logp -= logp.max()
    p = np.exp(logp)
    return p / p.sum()


def ideal_lambda(problem, state):
    kT = problem.kT[state // problem.M]
    mu = problem.mu[state % problem.M]
    lam_th = problem.lambda0 / math.sqrt(kT)
    return problem.volume * math.exp(mu / kT) / lam_th ** 3


def batch_means(orc, n_batches, sweeps_per_batch, exchange_every):
    """Run the oracle in batches; return per-batch, per-state mean N and mean E."""
    S = orc.p.S
    nb = np.zeros((n_batches, S))
    eb = np.zeros((n_batches, S))
    nvals = np.arange(orc.p.nmax + 1)
    for b in range(n_batches):
        h0, m0, o0 = orc.hN.copy(), orc.moments.copy(), orc.omega.copy()
        orc.run(sweeps_per_batch, exchange_every=exchange_every)
        dh = orc.hN - h0
        cnt = dh.sum(axis=1)
        nb[b] = (dh @ nvals) / np.maximum(cnt, 1)
        eb[b] = (orc.moments[:, 2] - m0[:, 2]) / np.maximum(orc.omega - o0, 1)
    return nb, eb


def zscores(batch, expected, sd_expected, n_obs):
    mean = batch.mean(axis=0)
    se = batch.std(axis=0, ddof=1) / math.sqrt(batch.shape[0])
    se = np.maximum(se, np.asarray(sd_expected) / math.sqrt(n_obs))
    se = np.maximum(se, 1e-12)
    return (mean - expected) / se


# ------------------------------------------------------------ pin functions

def pin_ideal_gas(mutation=0, exchange=False, n_batches=16, sweeps=250):
    """Max |z| of <N> per state against the truncated Poisson mean."""
    p = W.ideal_gas(W.fcc100_small())
    if exchange:
        # few grand-canonical moves between swaps, so that a wrong swap rule
        # cannot be washed out by the insertion/removal moves
        p = p.replace(moves_per_sweep=3, p_disp=0.0)
    orc = O.Oracle(p, mutation=mutation)
    nb, _ = batch_means(orc, n_batches, sweeps, exchange_every=1 if exchange else 0)
    exp_mean = np.zeros(p.S)
    exp_sd = np.zeros(p.S)
    nv = np.arange(p.nmax + 1)
    for s in range(p.S):
        pr = trunc_poisson(ideal_lambda(p, s), p.nmax)
        exp_mean[s] = pr @ nv
        exp_sd[s] = math.sqrt(pr @ nv ** 2 - exp_mean[s] ** 2)
    z = zscores(nb, exp_mean, exp_sd, n_batches * sweeps)
    return float(np.max(np.abs(z)))


def lj_np(r2, eps, sig, rc):
    s6 = (sig * sig / r2) ** 3
    return np.where(r2 < rc * rc, 4.0 * eps * (s6 * s6 - s6), 0.0)


def small_box_problem():
    """5.2 x 5.2 box, 4 surface atoms at z = 0, gas region 1.0 <= z <= 3.0,
    rc = 2.5, Nmax = 2, a 2 x 2 (kT, mu) grid."""
    surf = W.f32(np.array([[0.0, 0.0, 0.0], [2.6, 0.0, 0.0], [0.0, 2.6, 0.0], [2.6, 2.6, 0.0]]))
    eps = np.zeros((4, 4))
    sig = np.ones((4, 4))
    eps[0, 0] = 1.0
    eps[0, 1] = eps[1, 0] = 1.5
    return W.Problem(
        n_types=2, eps=eps, sigma=sig, rc=2.5, Lx=5.2, Ly=5.2, Lz=3.0, periodic_z=0,
        z_lo=1.0, z_hi=3.0, surf_xyz=surf, surf_type=np.ones(4, np.int32),
        kT=np.array([0.9, 1.3]), mu=np.array([-5.5, -4.0]), lambda0=1.0, nmax=2,
        moves_per_sweep=20, max_disp=0.4, p_disp=1.0 / 3.0, seed=7,
        e_lo=-40.0, e_bin=0.05, n_e_bins=1600, name="small_box")


def e_surf_np(p, pts):
    e = np.zeros(len(pts))
    for a in p.surf_xyz:
        d = pts - a
        d[:, 0] -= p.Lx * np.round(d[:, 0] / p.Lx)
        d[:, 1] -= p.Ly * np.round(d[:, 1] / p.Ly)
        e += lj_np(np.sum(d * d, axis=1), p.eps[0, 1], p.sigma[0, 1], p.rc)
    return e


def brute_force_small_box(p, n_grid=(64, 64, 40), n_mc=1_500_000, seed=11):
    """P(N) and <E> for N <= 2 per temperature of the small box.

    Z_1(beta) = int g, g = exp(-beta e_s), by the midpoint rule;
    Z_2 = Z_1^2 + int int g1 g2 (exp(-beta phi12) - 1), the second term (the
    Mayer part, zero for r12 >= rc) by Monte Carlo with r2 = r1 + d, d uniform
    in the cutoff ball.  Returns {kT: (Z1, Z2, E1, E2)}, E_N = <E | N>."""
    nx, ny, nz = n_grid
    hx, hy, hz = p.Lx / nx, p.Ly / ny, (p.z_hi - p.z_lo) / nz
    gx = (np.arange(nx) + 0.5) * hx
    gy = (np.arange(ny) + 0.5) * hy
    gz = p.z_lo + (np.arange(nz) + 0.5) * hz
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")
    grid = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    es_grid = e_surf_np(p, grid)
    dv = hx * hy * hz
    rng = np.random.default_rng(seed)
    V = p.volume
    vball = 4.0 / 3.0 * math.pi * p.rc ** 3
    r1 = np.stack([rng.uniform(0, p.Lx, n_mc), rng.uniform(0, p.Ly, n_mc),
                   rng.uniform(p.z_lo, p.z_hi, n_mc)], axis=1)
    d = rng.normal(size=(n_mc, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    d *= (p.rc * rng.uniform(0, 1, n_mc) ** (1.0 / 3.0))[:, None]
    r2 = r1 + d
    inside = (r2[:, 2] >= p.z_lo) & (r2[:, 2] <= p.z_hi)
    r2[:, 0] %= p.Lx
    r2[:, 1] %= p.Ly
    e1 = e_surf_np(p, r1)
    e2 = e_surf_np(p, r2)
    phi = lj_np(np.sum(d * d, axis=1), p.eps[0, 0], p.sigma[0, 0], p.rc)
    out = {}
    for kT in p.kT:
        b = 1.0 / kT
        g = np.exp(-b * es_grid)
        z1 = g.sum() * dv
        i1 = (es_grid * g).sum() * dv
        gg = np.exp(-b * (e1 + e2)) * inside
        mayer = V * vball * np.mean(gg * (np.exp(-b * phi) - 1.0))
        emayer = V * vball * np.mean(gg * (np.exp(-b * phi) * (e1 + e2 + phi) - (e1 + e2)))
        z2 = z1 * z1 + mayer
        out[float(kT)] = (z1, z2, i1 / z1, (2.0 * z1 * i1 + emayer) / z2)
    return out


def pin_small_box(mutation=0, n_batches=16, sweeps=3000):
    """Max |z| of <N> and <E> per state against the brute-force values."""
    p = small_box_problem()
    bf = brute_force_small_box(p)
    exp_n, exp_e, sd_n, sd_e = (np.zeros(p.S) for _ in range(4))
    for s in range(p.S):
        kT = p.kT[s // p.M]
        mu = p.mu[s % p.M]
        z1, z2, e1, e2 = bf[float(kT)]
        zz = math.exp(mu / kT) / (p.lambda0 / math.sqrt(kT)) ** 3
        w = np.array([1.0, zz * z1, zz * zz * z2 / 2.0])
        w /= w.sum()
        exp_n[s] = w @ np.arange(3)
        sd_n[s] = math.sqrt(w @ np.arange(3) ** 2 - exp_n[s] ** 2)
        exp_e[s] = w[1] * e1 + w[2] * e2
        sd_e[s] = 1.0
    orc = O.Oracle(p, mutation=mutation)
    orc.run(500, exchange_every=10, hist=False)
    nb, eb = batch_means(orc, n_batches, sweeps, exchange_every=10)
    zn = zscores(nb, exp_n, sd_n, n_batches * sweeps)
    ze = zscores(eb, exp_e, sd_e, n_batches * sweeps)
    return float(max(np.max(np.abs(zn)), np.max(np.abs(ze))))


def dense_walkers(seed=3):
    p = W.fcc100_small()
    pos, n = W.initial_walkers(p, [24] * p.S, seed=seed)
    return p, pos, n


def pin_incremental_energy(mutation=0):
    """Max |E_running - E_recomputed| after a run at high density."""
    p, pos, n = dense_walkers()
    orc = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    orc.run(200, exchange_every=10, hist=False)
    err = [abs(orc.energy[w] - orc.total_energy(w)) for w in range(p.S)]
    return float(max(err))


def pin_image_sum(mutation=0):
    """Max |particle energy - explicit periodic-image sum|."""
    p, pos, n = dense_walkers(seed=5)
    orc = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    rng = np.random.default_rng(1)
    worst = 0.0
    for w in range(4):
        for _ in range(20):
            q = np.array([rng.uniform(0, p.Lx), rng.uniform(0, p.Ly), rng.uniform(p.z_lo, p.z_hi)])
            e, _, _, _ = orc.particle_energy(w, q)
            ref = 0.0
            others = [(a, 1) for a in p.surf_xyz] + [(pos[w, j], 0) for j in range(n[w])]
            for r, t in others:
                for ix in (-1, 0, 1):
                    for iy in (-1, 0, 1):
                        d = q - (r + np.array([ix * p.Lx, iy * p.Ly, 0.0]))
                        ref += orc.phi(0, t, float(d @ d))
            worst = max(worst, abs(e - ref))
    return worst


def log_density(p, state, n, energy):
    """ln of Eq. Ngrand at state s for a configuration with n particles and
    energy E (scaled coordinates, so that V^N stays in the density)."""
    kT = p.kT[state // p.M]
    mu = p.mu[state % p.M]
    lam = p.lambda0 / math.sqrt(kT)
    return (mu / kT) * n + n * math.log(p.volume) - 3 * n * math.log(lam) \
        - math.lgamma(n + 1) - energy / kT


def pin_acceptance_ratios(mutation=0):
    """Max |log alpha - ln density ratio| over random moves and swaps."""
    p = W.fcc100_small()
    orc = O.Oracle(p, mutation=mutation)
    rng = np.random.default_rng(2)
    worst = 0.0
    for _ in range(200):
        s = int(rng.integers(p.S))
        n = int(rng.integers(1, p.nmax))
        e0 = rng.normal() * 5
        de = rng.normal() * 3
        ins = log_density(p, s, n + 1, e0 + de) - log_density(p, s, n, e0)
        rem = log_density(p, s, n - 1, e0 + de) - log_density(p, s, n, e0)
        disp = log_density(p, s, n, e0 + de) - log_density(p, s, n, e0)
        worst = max(worst, abs(orc.log_alpha(1, s, n, de) - ins),
                    abs(orc.log_alpha(2, s, n, de) - rem), abs(orc.log_alpha(0, s, n, de) - disp))
        sa, sb = (int(x) for x in rng.choice(p.S, 2, replace=False))
        na, nb = (int(x) for x in rng.integers(0, p.nmax + 1, 2))
        ea, eb = rng.normal(size=2) * 10
        swap = (log_density(p, sa, nb, eb) + log_density(p, sb, na, ea)
                - log_density(p, sa, na, ea) - log_density(p, sb, nb, eb))
        worst = max(worst, abs(orc.exchange_log_alpha(sa, sb, na, nb, ea, eb) - swap))
    return worst


# ---------------------------------------------------------------- the tests

def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_pair_potential_closed_form_facts():
    p = W.fcc100_small()
    orc = O.Oracle(p)
    for t, (eps, sig) in {0: (1.0, 1.0), 1: (2.0, 1.0)}.items():
        assert abs(orc.phi(0, t, sig * sig)) < 1e-14                 # zero crossing at sigma
        rmin2 = (2 ** (1 / 6) * sig) ** 2
        assert abs(orc.phi(0, t, rmin2) + eps) < 1e-12               # well depth
        h = 1e-5
        d = (orc.phi(0, t, (2 ** (1 / 6) + h) ** 2) - orc.phi(0, t, (2 ** (1 / 6) - h) ** 2)) / (2 * h)
        assert abs(d) < 1e-6                                         # minimum location
        assert orc.phi(0, t, 2.5 ** 2) == 0.0                        # truncation: r >= rc
        assert orc.phi(0, t, 3.0 ** 2) == 0.0
        assert orc.phi(0, t, 2.4999 ** 2) < 0.0


def test_image_sum():
    assert pin_image_sum() < 1e-10


def test_incremental_energy_matches_recompute():
    assert pin_incremental_energy() < 1e-8


def test_acceptance_ratios_are_density_ratios():
    assert pin_acceptance_ratios() < 1e-9


def test_ideal_gas_truncated_poisson():
    assert pin_ideal_gas() < 4.5


def test_ideal_gas_with_replica_exchange():
    assert pin_ideal_gas(exchange=True) < 4.5


@pytest.mark.slow
def test_small_box_brute_force():
    assert pin_small_box() < 4.5


def test_swap_of_identical_states_always_accepted():
    p = W.fcc100_small(L=1, M=2).replace(mu=np.array([-3.0, -3.0]))
    orc = O.Oracle(p)
    assert orc.exchange_log_alpha(0, 1, 5, 9, -3.0, -40.0) == pytest.approx(0.0, abs=1e-12)


# which pins must catch each planted mistake (see regc_oracle.c for the bits)
CATCHERS = {
    1: ["acceptance", "ideal+RE"],        # mu-term sign in the swap rule
    2: ["acceptance", "ideal+RE"],        # Lambda factor of the swap rule
    4: ["acceptance", "ideal", "small_box"],   # Lambda^1 for Lambda^3
    8: ["acceptance", "ideal", "small_box"],   # 1/(N+1) dropped
    16: ["lj", "small_box"],              # factor 4 of the LJ potential
    32: ["images"],                        # no minimum image along y
    64: ["incremental"],                   # removes another particle than it priced
}


def _pin_fails(name, bit):
    if name == "acceptance":
        return pin_acceptance_ratios(bit) > 1e-9
    if name == "images":
        return pin_image_sum(bit) > 1e-10
    if name == "incremental":
        return pin_incremental_energy(bit) > 1e-8
    if name == "lj":
        orc = O.Oracle(W.fcc100_small(), mutation=bit)
        return abs(orc.phi(0, 0, 2 ** (1 / 3)) + 1.0) > 1e-12
    if name == "ideal":
        return pin_ideal_gas(bit, n_batches=8, sweeps=150) > 6
    if name == "ideal+RE":
        return pin_ideal_gas(bit, exchange=True, n_batches=8, sweeps=150) > 6
    if name == "small_box":
        return pin_small_box(bit, n_batches=8, sweeps=1500) > 6
    raise KeyError(name)


@pytest.mark.slow
@pytest.mark.parametrize("bit", sorted(CATCHERS))
def test_pins_detect_planted_mistakes(bit):
    """Each planted mistake makes every pin meant to catch it fail."""
    missed = [name for name in CATCHERS[bit] if not _pin_fails(name, bit)]
    assert not missed, "planted mistake %d went undetected by %s" % (bit, missed)
