"""GPU statistics and MBAR parity.

* The GPU sampler in the ideal-gas limit reproduces the truncated Poisson
  distribution of Eq. Ngrand at every state, with replica exchange on.
* On the 16-replica fcc(100) workload, per-state <N> and <E> of the GPU run
  agree with those of an independent FP64 oracle run within 3 combined
  standard errors (batch means over 50 batches of 2000 sweeps: shorter
  batches of this system are correlated, lag-1 about 0.65 at 200 sweeps, and
  would understate the errors), and the error of each is reported.
* The device MBAR solve and query (FP64 log-sum-exp) agree with the numpy
  oracle on seeded pooled histograms to 1e-9, and the handle's reweighting
  (histogram compaction + solve + query) agrees with the stand-alone entry
  points on the same histogram.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mbar as OM
from oracle import oracle as O
from paper_1908_11118_gb300 import Regc, mbar_last_info, mbar_query, mbar_solve
from paper_1908_11118_gb300.regc import mbar_solve_static
from paper_1908_11118_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def trunc_poisson(lam, nmax):
    n = np.arange(nmax + 1)
    lp = n * math.log(lam) - np.array([math.lgamma(k + 1) for k in n])
    p = np.exp(lp - lp.max())
    return p / p.sum()


def batches_gpu(g, n_batches, sweeps, exchange_every):
    S = g.S
    nb, eb = np.zeros((n_batches, S)), np.zeros((n_batches, S))
    nv = np.arange(g.nmax + 1)
    prev = g.histograms()
    for b in range(n_batches):
        g.run(sweeps, exchange_every=exchange_every)
        h = g.histograms()
        dh = h["hN"] - prev["hN"]
        nb[b] = (dh @ nv) / np.maximum(dh.sum(axis=1), 1)
        eb[b] = (h["moments"][:, 2] - prev["moments"][:, 2]) / np.maximum(h["omega"] - prev["omega"], 1)
        prev = h
    return nb, eb


def batches_oracle(o, n_batches, sweeps, exchange_every):
    S = o.p.S
    nb, eb = np.zeros((n_batches, S)), np.zeros((n_batches, S))
    nv = np.arange(o.p.nmax + 1)
    for b in range(n_batches):
        h0, m0, om0 = o.hN.copy(), o.moments.copy(), o.omega.copy()
        o.run(sweeps, exchange_every=exchange_every)
        dh = o.hN - h0
        nb[b] = (dh @ nv) / np.maximum(dh.sum(axis=1), 1)
        eb[b] = (o.moments[:, 2] - m0[:, 2]) / np.maximum(o.omega - om0, 1)
    return nb, eb


def mean_se(x):
    return x.mean(axis=0), x.std(axis=0, ddof=1) / math.sqrt(x.shape[0])


def test_gpu_ideal_gas_with_exchange():
    p = W.ideal_gas(W.fcc100_small()).replace(moves_per_sweep=3, p_disp=0.0)
    g = Regc(p)
    nb, _ = batches_gpu(g, 50, 400, exchange_every=1)
    m, se = mean_se(nb)
    nv = np.arange(p.nmax + 1)
    for s in range(p.S):
        kT, mu = p.kT[s // p.M], p.mu[s % p.M]
        pr = trunc_poisson(p.volume * math.exp(mu / kT) * kT ** 1.5, p.nmax)
        mean = pr @ nv
        sd = math.sqrt(pr @ nv ** 2 - mean ** 2)
        err = max(se[s], sd / math.sqrt(50 * 400))
        assert abs(m[s] - mean) < 3.0 * err, (s, m[s], mean, err)


def test_statistical_parity_with_oracle_fcc100():
    """<N> and <E> per state: 16 replicas, 1000 + 50 x 2000 sweeps of 20 moves,
    exchange every 10 sweeps, GPU and oracle each from N = 0 (their chains are
    independent: the oracle's seed differs)."""
    p = W.fcc100_small()
    g = Regc(p)
    o = O.Oracle(p.replace(seed=1))
    g.run(1000)
    o.run(1000, hist=False)
    gn, ge = batches_gpu(g, 50, 2000, 10)
    on, oe = batches_oracle(o, 50, 2000, 10)
    gm, gs = mean_se(gn)
    om, os_ = mean_se(on)
    gem, ges = mean_se(ge)
    oem, oes = mean_se(oe)
    zn = np.abs(gm - om) / np.maximum(np.hypot(gs, os_), 1e-3)
    ze = np.abs(gem - oem) / np.maximum(np.hypot(ges, oes), 1e-3)
    print("max z <N> %.2f, <E> %.2f; SE(<N>) gpu %.3g oracle %.3g" % (zn.max(), ze.max(), gs.max(), os_.max()))
    for s in range(p.S):
        print("state %2d  <N> gpu %.4f oracle %.4f (SE %.4f, %.4f)  <E> gpu %.4f oracle %.4f (SE %.4f, %.4f)"
              % (s, gm[s], om[s], gs[s], os_[s], gem[s], oem[s], ges[s], oes[s]))
    assert zn.max() < 3.0 and ze.max() < 3.0
    assert g.check_energy() == 0.0


def synthetic_bins(seed=0, S_side=5, nmax=30, kT_range=(0.7, 1.6), mu_range=(-5.0, -2.0), per_n=40):
    """Seeded pooled (N, E) histogram drawn from a model density of states."""
    rng = np.random.default_rng(seed)
    kT = np.repeat(np.geomspace(*kT_range, S_side), S_side)
    mu = np.tile(np.linspace(*mu_range, S_side), S_side)
    N = np.repeat(np.arange(nmax + 1), per_n)
    E = -2.5 * N + rng.normal(size=N.size) * (1.0 + 0.3 * np.sqrt(N))
    E = np.round(E * 20.0) / 20.0
    lnw_s = (-(E[None, :] - mu[:, None] * N[None, :]) / kT[:, None]
             + N[None, :] * (1.5 * np.log(kT)[:, None] + math.log(300.0))
             - np.array([math.lgamma(k + 1) for k in N])[None, :])
    omega = rng.integers(500, 3000, len(kT)).astype(float)
    H = np.zeros(N.size)
    for s in range(len(kT)):
        w = np.exp(lnw_s[s] - lnw_s[s].max())
        H += omega[s] * w / w.sum()
    keep = H > 1e-3
    return kT, mu, omega, N[keep], E[keep], H[keep], nmax


def test_mbar_solve_and_query_match_oracle():
    kT, mu, omega, N, E, H, nmax = synthetic_bins()
    f_o, D_o, it_o, ok = OM.solve(kT, mu, 1.0, omega, N, E, H, tol=1e-11)
    assert ok
    f_g, D_g, it_g = mbar_solve(kT, mu, 1.0, omega, N, E, H, tol=1e-11)
    np.testing.assert_allclose(f_g, f_o, atol=1e-9)
    np.testing.assert_allclose(D_g, D_o, atol=1e-9)
    assert it_g <= it_o           # the same fixed point, reached by an accelerated iteration
    kq = np.array([0.75, 1.0, 1.2, 1.55])
    mq = np.array([-4.5, -3.3, -2.7, -2.2])
    n_o, p_o, fq_o = OM.query(kq, mq, 1.0, N, E, H, D_o, nmax)
    n_g, p_g, fq_g = mbar_query(kq, mq, 1.0, N, E, H, D_g, nmax)
    np.testing.assert_allclose(n_g, n_o, rtol=1e-9)
    np.testing.assert_allclose(p_g, p_o, atol=1e-10)
    np.testing.assert_allclose(fq_g, fq_o, atol=1e-9)


def test_sparse_kernel_matrix_solves_the_oracle_equations():
    """64 well separated states over N <= 300: most of the kernel matrix lies
    more than e^-70 below its bin's largest term and is dropped.  The device
    solution is a fixed point of the oracle's own map (one FP64 map from it
    moves f by < 1e-9, and gives the same D_b), and it agrees with the
    log-sum-exp solve of the allocation-free entry point."""
    kT, mu, omega, N, E, H, nmax = synthetic_bins(seed=5, S_side=8, nmax=300, kT_range=(0.5, 1.6),
                                                  mu_range=(-6.0, -1.0), per_n=12)
    f_g, D_g, it_g = mbar_solve(kT, mu, 1.0, omega, N, E, H, tol=1e-12)
    info = mbar_last_info()
    S, B = len(kT), len(N)
    assert info["path"] == 1 and info["builds"] >= 1 and (info["S"], info["B"]) == (S, B)
    assert 0 < info["nnz"] < 0.5 * S * B, info
    f1, D1, _, _ = OM.solve(kT, mu, 1.0, omega, N, E, H, max_iter=1, f0=f_g)
    np.testing.assert_allclose(f1, f_g, atol=1e-9)
    np.testing.assert_allclose(D_g, D1, atol=1e-9)
    f_s, D_s, _ = mbar_solve_static(kT, mu, 1.0, omega, N, E, H, tol=1e-12)
    assert mbar_last_info()["path"] == 0
    np.testing.assert_allclose(f_g, f_s, atol=1e-8)
    np.testing.assert_allclose(D_g, D_s, atol=1e-8)


@pytest.fixture(scope="module")
def fcc111_run():
    """The 1024-replica fcc(111) workload (Nmax 512) after 2000 + 20000 sweeps."""
    p = W.fcc111_paper_scale(seed=0)
    rng = np.random.default_rng(0)
    pos, n = W.lattice_walkers(p, rng.integers(0, p.nmax // 2 + 1, p.S), seed=0)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.run(2000)
    g.reset_histograms()
    g.run(20000)
    yield p, g, g.histograms()
    g.close()


def test_full_size_solve_satisfies_sampled_equations(fcc111_run):
    """The device solve over the full-size run's pooled bins (about 1e6 of
    them, on the sparse kernel matrix) satisfies, checked one by one in FP64
    by the oracle's reduced potential, the D equation
        D_b = ln sum_k Omega_k exp(f_k - u_k(b))
    at 200 sampled bins and the f equation
        f_s - f_0 = -ln sum_b H_b exp(-u_s(b) - D_b) + ln sum_b H_b exp(-u_0(b) - D_b)
    at 24 sampled states."""
    p, _, h = fcc111_run
    rng = np.random.default_rng(1)
    N_b, E_b, H_b = OM.occupied_bins(h["hNE"], p.e_lo, p.e_bin)
    kT_s, mu_s = np.repeat(p.kT, p.M), np.tile(p.mu, p.L)
    omega = h["omega"].astype(float)
    f, D, it = mbar_solve(kT_s, mu_s, p.lambda0, omega, N_b, E_b, H_b, tol=1e-10, max_iter=200000)
    info = mbar_last_info()
    S, B = p.S, len(N_b)
    assert info["path"] == 1 and info["nnz"] < 0.5 * S * B, info
    assert B > 200000
    sb = np.sort(rng.choice(B, 200, replace=False))
    u = OM.reduced_potential(kT_s, mu_s, p.lambda0, N_b[sb], E_b[sb])           # [S, 200]
    D_o = OM.lse(np.log(omega)[:, None] + f[:, None] - u, axis=0)
    np.testing.assert_allclose(D[sb], D_o, rtol=0, atol=1e-9)
    ss = np.concatenate([[0], np.sort(rng.choice(np.arange(1, S), 23, replace=False))])
    u = OM.reduced_potential(kT_s[ss], mu_s[ss], p.lambda0, N_b, E_b)          # [24, B]
    f_o = -OM.lse(np.log(H_b)[None, :] - u - D[None, :], axis=1)
    np.testing.assert_allclose(f_o - f_o[0], f[ss], rtol=0, atol=1e-8)


def test_warm_started_handle_reweight_reaches_the_same_fixed_point(fcc111_run):
    """The handle's reweighting starts the full-size problem from the solve
    with 16 energy bins merged; it reaches the fixed point the cold solve of
    the same bins reaches, with fewer matrix builds."""
    p, g, h = fcc111_run
    N_b, E_b, H_b = OM.occupied_bins(h["hNE"], p.e_lo, p.e_bin)
    kT_s, mu_s = np.repeat(p.kT, p.M), np.tile(p.mu, p.L)
    f_c, _, _ = mbar_solve(kT_s, mu_s, p.lambda0, h["omega"].astype(float), N_b, E_b, H_b, tol=1e-11,
                           max_iter=200000)
    cold = mbar_last_info()
    kq, mq = np.array([0.8, 1.2]), np.array([-4.0, -3.0])
    _, _, f_w, _ = g.reweight(kq, mq, tol=1e-11, max_iter=200000)
    warm = mbar_last_info()
    assert warm["coarse_B"] > 0 and warm["coarse_B"] * 4 <= warm["B"] and warm["coarse_iterations"] > 0
    assert cold["coarse_B"] == 0 and warm["builds"] < cold["builds"], (warm, cold)
    np.testing.assert_allclose(f_w, f_c, rtol=0, atol=1e-7)


def test_handle_reweight_matches_standalone_entry_points():
    """regc_reweight (device compaction of the pooled histogram, solve, query)
    gives what regc_mbar_solve / regc_mbar_query give on the same bins."""
    p = W.fcc100_small()
    g = Regc(p)
    g.run(600)
    h = g.histograms()
    kq = np.array([0.7, 1.0, 1.3])
    mq = np.array([-5.0, -3.5, -2.5])
    n_h, p_h, f_h, it = g.reweight(kq, mq, tol=1e-10)
    n_idx, k_idx = np.nonzero(h["hNE"])
    N_b = n_idx.astype(np.int32)
    E_b = p.e_lo + (k_idx + 0.5) * p.e_bin
    H_b = h["hNE"][n_idx, k_idx].astype(float)
    kT_s = np.repeat(p.kT, p.M)
    mu_s = np.tile(p.mu, p.L)
    f_s, D_s, it_s = mbar_solve(kT_s, mu_s, p.lambda0, h["omega"].astype(float), N_b, E_b, H_b, tol=1e-10)
    n_s, p_s, _ = mbar_query(kq, mq, p.lambda0, N_b, E_b, H_b, D_s, p.nmax)
    assert it == it_s
    np.testing.assert_allclose(f_h, f_s, atol=1e-12)
    np.testing.assert_allclose(n_h, n_s, rtol=1e-12)
    np.testing.assert_allclose(p_h, p_s, atol=1e-12)
