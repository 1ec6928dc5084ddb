"""Pins of the surrogate and delayed-acceptance oracle.

* Analytic gradients of the MSE loss against central finite differences.
* Features against closed forms: a neighbour exactly at a centre gives that
  Gaussian the value of the cutoff function; its two neighbours get
  exp(-1/2) of it; a neighbour at rc contributes nothing; contributions add.
* The C oracle's features and network output agree with the numpy ones.
* Adam's first step moves every parameter by lr against the sign of its gradient.
* Delayed acceptance with arbitrary (random, untrained) weights still samples
  the distribution of Eq. Ngrand: the ideal-gas truncated Poisson limit and the
  brute-force partition functions of the small box.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from oracle import surrogate as SG
from test_oracle_pins import (batch_means, brute_force_small_box, ideal_lambda, small_box_problem,
                              trunc_poisson, zscores)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = SG.init_params(1, scale=0.7)
    X = rng.uniform(0, 3, size=(12, 16))
    y = rng.normal(size=12)
    loss, g = SG.loss_and_grad(theta, X, y)
    idx = rng.choice(SG.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [SG.N_PARAMS - 1, 0, 16 * 64 + 3]])
    for i in idx:
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (SG.loss_and_grad(tp, X, y)[0] - SG.loss_and_grad(tm, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, i


def test_features_closed_forms():
    rc = 2.5
    for k in (2, 7, 12):
        c = SG.CENTRES[k]
        f = SG.features([c], [1.0], rc)
        fc = 0.5 * (math.cos(math.pi * c / rc) + 1)
        assert f[k] == pytest.approx(fc, rel=1e-14)
        assert f[k - 1] == pytest.approx(fc * math.exp(-0.5), rel=1e-12)
        assert f[k + 1] == pytest.approx(fc * math.exp(-0.5), rel=1e-12)
    assert np.all(SG.features([rc], [2.0], rc) == 0.0)
    a = SG.features([1.1], [1.0], rc)
    b = SG.features([1.7], [2.0], rc)
    np.testing.assert_allclose(SG.features([1.1, 1.7], [1.0, 2.0], rc), a + b, rtol=1e-14)
    assert np.all(SG.features([1.7], [2.0], rc) == pytest.approx(2 * SG.features([1.7], [1.0], rc)))


def test_c_oracle_features_and_network_agree_with_numpy():
    p = W.fcc100_small(L=1, M=1)
    pos, n = W.initial_walkers(p, 20, seed=3)
    theta = SG.to_bf16(SG.init_params(4))
    orc = O.Oracle(p, pos=pos, n=n, surrogate=theta)
    rng = np.random.default_rng(5)
    for _ in range(10):
        q = np.array([rng.uniform(0, p.Lx), rng.uniform(0, p.Ly), rng.uniform(p.z_lo, p.z_lo + 3)])
        e, feat = orc.surrogate_energy(0, q)
        pts = np.concatenate([p.surf_xyz, pos[0, :n[0]]])
        w = np.concatenate([np.full(p.n_surf, p.eps[0, 1]), np.full(n[0], p.eps[0, 0])])
        d = q - pts
        d[:, 0] -= p.Lx * np.round(d[:, 0] / p.Lx)
        d[:, 1] -= p.Ly * np.round(d[:, 1] / p.Ly)
        r = np.sqrt(np.sum(d * d, axis=1))
        ref = SG.features(r, w, p.rc)
        np.testing.assert_allclose(feat, ref, rtol=1e-12, atol=1e-14)
        # the sampler's network: bfloat16 weights and layer inputs
        e_ref, _ = SG.forward(theta, ref[None, :], bf16_inputs=True)
        assert e == pytest.approx(e_ref[0], rel=1e-12, abs=1e-12)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159, 1e-3])
    b = SG.to_bf16(x)
    bits = b.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert b[0] == 1.0
    assert b[1] == 1.0                     # halfway between 1 and 1 + 2^-7: ties to even
    assert b[2] == 1.0                     # below halfway
    assert b[3] == 1.0 + 2 ** -7           # above halfway
    assert np.all(np.abs(b - x) <= np.abs(x) * 2 ** -8)


def test_adam_first_step_is_lr_times_sign():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    opt = SG.Adam(3, lr=0.01)
    new = opt.step(theta, g)
    np.testing.assert_allclose(new, theta - 0.01 * np.sign(g), rtol=1e-6)


def pin_da_ideal_gas(theta, n_batches=16, sweeps=250):
    p = W.ideal_gas(W.fcc100_small()).replace(moves_per_sweep=3, p_disp=0.0)
    orc = O.Oracle(p, surrogate=theta)
    nb, _ = batch_means(orc, n_batches, sweeps, exchange_every=1)
    nv = np.arange(p.nmax + 1)
    exp_mean, exp_sd = np.zeros(p.S), np.zeros(p.S)
    for s in range(p.S):
        pr = trunc_poisson(ideal_lambda(p, s), p.nmax)
        exp_mean[s] = pr @ nv
        exp_sd[s] = math.sqrt(pr @ nv ** 2 - exp_mean[s] ** 2)
    return float(np.max(np.abs(zscores(nb, exp_mean, exp_sd, n_batches * sweeps))))


def test_planted_da_mistake_is_detected():
    """Stage 2 without the -dE~ correction biases the chain (oracle bit 128)."""
    theta = SG.to_bf16(SG.init_params(9, scale=1.5))
    theta[-1] = 0.7
    p = W.ideal_gas(W.fcc100_small()).replace(moves_per_sweep=3, p_disp=0.0)
    orc = O.Oracle(p, surrogate=theta, mutation=128)
    nb, _ = batch_means(orc, 8, 150, exchange_every=1)
    nv = np.arange(p.nmax + 1)
    means = np.array([trunc_poisson(ideal_lambda(p, s), p.nmax) @ nv for s in range(p.S)])
    assert np.max(np.abs(nb.mean(axis=0) - means)) > 1.0


def test_delayed_acceptance_ideal_gas_any_weights():
    # with eps = 0 every feature is zero, so e~ is a constant c of the network
    # (the output bias makes it non-zero): insertions see dE~ = c and removals
    # -c, a screen that favours one direction; the chain must stay exact
    theta = SG.to_bf16(SG.init_params(9, scale=1.5))
    theta[-1] = 0.7
    assert pin_da_ideal_gas(theta) < 4.5


@pytest.mark.slow
def test_delayed_acceptance_small_box_brute_force():
    p = small_box_problem()
    bf = brute_force_small_box(p)
    theta = SG.to_bf16(SG.init_params(2, scale=1.0))
    orc = O.Oracle(p, surrogate=theta)
    orc.run(500, exchange_every=10, hist=False)
    nb, eb = batch_means(orc, 16, 3000, exchange_every=10)
    exp_n, sd_n, exp_e = np.zeros(p.S), np.zeros(p.S), np.zeros(p.S)
    for s in range(p.S):
        kT, mu = p.kT[s // p.M], p.mu[s % p.M]
        z1, z2, e1, e2 = bf[float(kT)]
        zz = math.exp(mu / kT) / (p.lambda0 / math.sqrt(kT)) ** 3
        w = np.array([1.0, zz * z1, zz * zz * z2 / 2.0])
        w /= w.sum()
        exp_n[s] = w @ np.arange(3)
        sd_n[s] = math.sqrt(w @ np.arange(3) ** 2 - exp_n[s] ** 2)
        exp_e[s] = w[1] * e1 + w[2] * e2
    zn = zscores(nb, exp_n, sd_n, 16 * 3000)
    ze = zscores(eb, exp_e, np.ones(p.S), 16 * 3000)
    assert max(np.max(np.abs(zn)), np.max(np.abs(ze))) < 4.5
    # the surrogate screened: some moves were rejected at stage 1
    tr = orc.sweeps(20, trace=True)
    ev = tr["status"] == 0
    assert 0 < np.mean(tr["stage1"][ev]) < 1


def test_bf16_training_gradient_within_bfloat16_of_the_exact_one():
    """The mixed-precision gradient (bfloat16 operands of every matrix
    product) against the FP64 analytic gradient, itself pinned by finite
    differences: within a few bfloat16 roundings (2^-8) of the per-row
    gradient magnitudes.  A transposed or dropped operand is far outside."""
    rng = np.random.default_rng(3)
    th = SG.init_params(7)
    th[~SG.weight_mask()] = rng.normal(size=int((~SG.weight_mask()).sum())) * 0.2
    X = rng.uniform(0.0, 3.0, size=(200, 16))
    y = rng.normal(0.0, 2.0, size=200)
    loss_b, g_b = SG.loss_and_grad_bf16(th, X, y)
    loss_e, g_e = SG.loss_and_grad(th, X, y)
    gabs = np.zeros(SG.N_PARAMS)
    for i in range(len(y)):
        gabs += np.abs(SG.loss_and_grad(th, X[i:i + 1], y[i:i + 1])[1]) / len(y)
    rel = np.abs(g_b - g_e) / (gabs + 1e-12)
    assert np.max(rel) < 6 * 2.0 ** -8
    assert np.median(rel) < 2.0 ** -8
    assert abs(loss_b - loss_e) < 0.05 * loss_e
    # planted: W2 transposed in the backward product
    W1, b1, W2, b2, W3, b3 = SG.unpack(th)
    th_t = SG.pack(W1, b1, W2.T, b2, W3, b3)
    _, g_t = SG.loss_and_grad_bf16(th_t, X, y)
    _, g_te = SG.loss_and_grad(th, X, y)
    assert np.max(np.abs(g_t - g_te) / (gabs + 1e-12)) > 0.1


def test_batch_rows_are_uniform_multiply_shift():
    key = (0x1234, 0x5678)
    rows = SG.batch_rows(1, 4096, 1000, key)
    assert rows.min() >= 0 and rows.max() < 1000
    counts = np.bincount(rows, minlength=1000)
    # 4096 draws over 1000 rows: chi-square with 999 degrees of freedom
    chi2 = float(np.sum((counts - 4.096) ** 2 / 4.096))
    assert abs(chi2 - 999) < 6 * np.sqrt(2 * 999)
    assert not np.array_equal(rows, SG.batch_rows(2, 4096, 1000, key))
