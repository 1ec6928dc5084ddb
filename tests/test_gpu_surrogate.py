"""GPU parity of the learned surrogate and of the delayed-acceptance sweep.

Every test calls the library through its C ABI and compares with the FP64
oracle on identical seeded inputs:
  * features and network output e~ of arbitrary positions, with the same
    inference parameters (bfloat16 weights, binary32 biases) and bfloat16
    layer inputs on both sides (the GPU runs the layers on tensor cores);
  * the training loss and its gradient (the library's forward and backward
    kernels) against the oracle's analytic backward pass, over several CTAs of
    rows and a ragged tail;
  * harvested training rows (particles and Philox probe points) against the
    oracle's features and exact interaction energies;
  * the delayed-acceptance sweep against the oracle's, move by move: both
    stages' decisions, the surrogate and exact energy changes, final states
    and counters, on the fcc(100) workload and the edge cases of the plain
    sweep;
  * in the ideal-gas limit, delayed acceptance with an untrained network keeps
    the truncated Poisson distribution;
  * training on the GPU lowers the loss, and the trained network screens:
    fewer exact evaluations per accepted move than the plain sweep and than
    the untrained network, with <N> unchanged within the statistical error.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from oracle import surrogate as SG
from paper_1908_11118_gb300 import Regc, surrogate_gradient
from paper_1908_11118_gb300 import build as B
from parity import compare_da_traces
from test_gpu_parity import EDGE_CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    O.build()


def theta_of(seed, scale=1.0):
    """Seeded parameters with non-zero biases, as the sampler's network holds them."""
    th = SG.init_params(seed, scale)
    rng = np.random.default_rng(seed + 100)
    m = ~SG.weight_mask()
    th[m] = rng.normal(size=int(m.sum())) * 0.3
    return SG.inference_params(th)


# Tolerances of the binary32 surrogate against FP64:
# each feature term carries the error of the cosine cutoff (absolute, about
# 2^-21 of the weight) and of exp2 and the distance (a few ulp, relative), so
#   |dG_k| <= 4e-6 (sum of the weights within rc) + 1e-5 |G_k|;
# e~ then moves by at most sum_k |de~/dG_k| |dG_k| plus the rounding of three
# dot products, which the tests bound by 2e-4 (1 + |e~|).
def feat_tol(fo, wsum):
    return 4e-6 * wsum + 1e-5 * np.abs(fo) + 1e-7


def e_tol(eo):
    return 2e-4 * (1.0 + np.abs(eo))


def sur_tol_of(rec):
    # dE~ is one or two network outputs; the scale of each is bounded by
    # |dE~| + 2 max|e~| of the workload (below 40 for these networks)
    return 2e-4 * (2.0 + abs(rec["dE_sur"]) + 80.0)


def weight_sum(p, pos_w, n_w, q):
    """Sum of the neighbour weights eps_0j within rc of q (nearest image)."""
    pts = np.concatenate([p.surf_xyz, pos_w[:n_w]])
    w = np.concatenate([p.eps[0, np.asarray(p.surf_type)], np.full(n_w, p.eps[0, 0])])
    d = q[None, :] - pts
    d[:, 0] -= p.Lx * np.round(d[:, 0] / p.Lx)
    d[:, 1] -= p.Ly * np.round(d[:, 1] / p.Ly)
    if p.periodic_z:
        d[:, 2] -= p.Lz * np.round(d[:, 2] / p.Lz)
    r2 = np.sum(d * d, axis=1)
    return float(w[r2 < p.rc ** 2].sum())


def test_eval_matches_oracle():
    p = W.fcc100_small()
    pos, n = W.initial_walkers(p, np.arange(p.S) * 2 % 29, seed=3)
    th = theta_of(4)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.surrogate_set(th)
    o = O.Oracle(p, pos=pos, n=n, surrogate=th)
    rng = np.random.default_rng(1)
    worst_f, worst_e = 0.0, 0.0
    for w in (0, 5, 9, 15):
        q = np.stack([rng.uniform(0, p.Lx, 96), rng.uniform(0, p.Ly, 96),
                      rng.uniform(p.z_lo, p.z_hi, 96)], axis=1).astype(np.float32)
        e, f = g.surrogate_eval(w, q)
        for i in range(len(q)):
            qd = q[i].astype(np.float64)
            eo, fo = o.surrogate_energy(w, qd)
            ws = weight_sum(p, o.pos[w], int(o.n[w]), qd)
            tf = feat_tol(fo, ws)
            assert np.all(np.abs(f[i] - fo) <= tf), (w, i, f[i] - fo, tf)
            assert abs(e[i] - eo) <= e_tol(eo), (w, i, e[i], eo)
            worst_f = max(worst_f, float(np.max(np.abs(f[i] - fo) / tf)))
            worst_e = max(worst_e, abs(e[i] - eo) / e_tol(eo))
    print("worst feature error / tol %.3g, worst e~ error / tol %.3g" % (worst_f, worst_e))


def test_eval_empty_walker_and_far_from_surface():
    """With no neighbour within rc every feature is 0 and e~ is the network's
    value at G = 0: b3 + W3 . bf(silu(W2^T bf(silu(b1)) + b2)), bf the
    bfloat16 rounding of the layer inputs."""
    p = W.fcc100_small(L=1, M=1)
    th = theta_of(6)
    g = Regc(p)
    g.surrogate_set(th)
    q = np.array([[1.0, 2.0, p.z_hi - 0.1], [3.0, 0.5, p.z_hi]], np.float32)
    e, f = g.surrogate_eval(0, q)
    assert np.all(f == 0.0)
    W1, b1, W2, b2, W3, b3 = SG.unpack(th)
    bf = SG.to_bf16
    e0 = float(bf(SG.silu(bf(SG.silu(b1)) @ W2 + b2)) @ W3 + b3[0])
    assert np.all(np.abs(e - e0) <= e_tol(e0))


@pytest.mark.parametrize("n_rows", [1, 77, 128, 1000])
def test_gradient_matches_oracle(n_rows):
    rng = np.random.default_rng(n_rows)
    th = SG.init_params(7, scale=1.0).astype(np.float32)
    th[~SG.weight_mask()] = (rng.normal(size=int((~SG.weight_mask()).sum())) * 0.2).astype(np.float32)
    X = rng.uniform(0.0, 3.0, size=(n_rows, 16)).astype(np.float32)
    y = rng.normal(0.0, 2.0, size=n_rows).astype(np.float32)
    loss, grad = surrogate_gradient(th, X, y)
    th64, X64, y64 = th.astype(np.float64), X.astype(np.float64), y.astype(np.float64)
    loss_o, grad_o = SG.loss_and_grad(th64, X64, y64)
    # error scale: the sum over rows of each row's |gradient contribution|
    gabs = np.zeros(SG.N_PARAMS)
    for i in range(n_rows):
        gabs += np.abs(SG.loss_and_grad(th64, X64[i:i + 1], y64[i:i + 1])[1]) / n_rows
    tol = 3e-5 * gabs + 1e-9
    bad = np.abs(grad - grad_o) > tol
    assert not np.any(bad), (np.flatnonzero(bad)[:10], (np.abs(grad - grad_o) / tol).max())
    # loss = mean r^2 with r = e~ - y: each binary32 residual is off by at most
    # dr = 1e-5 (1 + |e~| + |y|), so the loss by mean(2 |r| dr + dr^2)
    e_o = SG.forward(th64, X64)[0]
    r = e_o - y64
    dr = 1e-5 * (1.0 + np.abs(e_o) + np.abs(y64))
    assert abs(loss - loss_o) <= float(np.mean(2 * np.abs(r) * dr + dr * dr)) + 1e-12


def grad_scale(th64, X64, y64):
    """Per parameter: the mean over rows of each row's |gradient contribution|."""
    gabs = np.zeros(SG.N_PARAMS)
    for i in range(len(y64)):
        gabs += np.abs(SG.loss_and_grad(th64, X64[i:i + 1], y64[i:i + 1])[1]) / len(y64)
    return gabs


@pytest.mark.parametrize("n_rows", [1, 77, 128, 1000])
def test_tensor_core_gradient_matches_oracle(n_rows):
    """The training gradient (BF16 operands on tensor cores, FP32
    accumulation) against the oracle's mixed-precision gradient with the same
    rounding points: the two differ by FP32 accumulation and SiLU, and by the
    rare operand that rounds to the neighbouring bfloat16 because its FP32 and
    FP64 values straddle the rounding point (one bfloat16 step, 2^-8, of one
    row's contribution).  Against the FP64 gradient: within a few bfloat16
    roundings of the per-row magnitudes."""
    rng = np.random.default_rng(n_rows + 11)
    th = SG.init_params(7, scale=1.0).astype(np.float32)
    th[~SG.weight_mask()] = (rng.normal(size=int((~SG.weight_mask()).sum())) * 0.2).astype(np.float32)
    X = rng.uniform(0.0, 3.0, size=(n_rows, 16)).astype(np.float32)
    y = rng.normal(0.0, 2.0, size=n_rows).astype(np.float32)
    loss, grad = surrogate_gradient(th, X, y, tensor_cores=True)
    th64, X64, y64 = th.astype(np.float64), X.astype(np.float64), y.astype(np.float64)
    loss_b, grad_b = SG.loss_and_grad_bf16(th64, X64, y64)
    loss_e, grad_e = SG.loss_and_grad(th64, X64, y64)
    gabs = grad_scale(th64, X64, y64)
    tol = 2e-4 * gabs + 2.0 ** -8 * gabs / np.sqrt(n_rows) + 1e-9
    ratio = np.abs(grad - grad_b) / tol
    print("worst |g - g_bf16 oracle| / tol %.3g; worst |g - g_fp64| / (sum |row g|) %.3g"
          % (ratio.max(), (np.abs(grad - grad_e) / (gabs + 1e-12)).max()))
    assert ratio.max() <= 1.0, np.flatnonzero(ratio > 1.0)[:10]
    if n_rows >= 64:
        # over many rows the BF16 roundings average out against the per-row
        # magnitudes; one row's gradient can cancel inside a contraction, where
        # no such relative bound holds
        assert np.max(np.abs(grad - grad_e) / (gabs + 1e-12)) < 6 * 2.0 ** -8
    assert abs(loss - loss_b) <= 1e-4 * (1.0 + loss_b)


def test_adam_steps_match_oracle():
    """Three Adam steps of regc_surrogate_train on caller rows against the
    oracle's Adam (FP64) on the oracle's mixed-precision gradient of the same
    mini-batches (Philox stream 6 draws the rows).  Adam's step
    lr m^/sqrt(v^) is a smooth function of the gradients away from zero: where
    every step's gradient of a parameter exceeds 20 times its tolerance
    (relative tolerance rel < 1/20), the update may differ from the oracle's
    by at most 3 rel lr per step; elsewhere the normalised step may point
    either way and is only bounded (|update| <= 3.2 lr per step)."""
    p = W.fcc100_small(L=2, M=2, seed=9)
    pos, n = W.initial_walkers(p, [20, 12, 26, 8], seed=4)
    o = O.Oracle(p, pos=pos, n=n, surrogate=theta_of(2))
    rng = np.random.default_rng(5)
    X, y = [], []
    for _ in range(600):
        w = int(rng.integers(p.S))
        q = np.array([rng.uniform(0, p.Lx), rng.uniform(0, p.Ly), rng.uniform(p.z_lo, p.z_lo + 4.0)])
        _, f = o.surrogate_energy(w, q)
        e, _, _, _ = o.particle_energy(w, q)
        X.append(f)
        y.append(min(e, 8.0))
    X = np.array(X, np.float32)
    y = np.array(y, np.float32)
    th = SG.init_params(3, scale=1.0).astype(np.float32)
    steps, batch, lr = 3, 256, 1e-3
    g = Regc(p)
    g.surrogate_set(th)
    g.surrogate_set_dataset(X, y, capacity=1024)
    losses = g.surrogate_train(steps, batch, lr)
    th_g = g.surrogate_get().astype(np.float64)
    key = (int(p.seed) & 0xFFFFFFFF, int(p.seed) >> 32)
    th_o = th.astype(np.float64)
    adam = SG.Adam(SG.N_PARAMS, lr)
    rel = np.zeros(SG.N_PARAMS)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    for a in range(1, steps + 1):
        rows = SG.batch_rows(a, batch, len(y), key)
        loss_o, grad_o = SG.loss_and_grad_bf16(th_o, X64[rows], y64[rows])
        assert abs(losses[a - 1] - loss_o) <= 1e-3 * (1.0 + loss_o)
        gs = grad_scale(th_o, X64[rows], y64[rows])
        gtol = 2e-4 * gs + 2.0 ** -8 * gs / np.sqrt(batch) + 1e-9
        rel = np.maximum(rel, gtol / np.maximum(np.abs(grad_o), 1e-300))
        th_o = adam.step(th_o, grad_o)
    d = np.abs(th_g - th_o)
    stable = rel < 0.05
    bound = 3.0 * rel * steps * lr + 1e-6 * np.abs(th_o)
    print("stable parameters %d of %d; worst |d theta| / bound (stable) %.3g; worst |d theta| / lr (other) %.3g"
          % (stable.sum(), SG.N_PARAMS, (d[stable] / bound[stable]).max(), d[~stable].max() / lr))
    assert stable.sum() > 0.5 * SG.N_PARAMS
    assert np.all(d[stable] <= bound[stable])
    assert np.all(d <= 3.2 * steps * lr)


def test_harvest_rows_match_oracle():
    p = W.fcc100_small()
    pos, n = W.initial_walkers(p, (np.arange(p.S) * 3) % 26, seed=5)
    g = Regc(p)
    g.set_walkers(pos, n)
    g.surrogate_set(theta_of(1))
    g.sweep(20)
    parts, probes = 3, 2
    clip = 4.0
    rows = g.surrogate_harvest(parts, probes, clip, capacity=p.S * (parts + probes) * 2)
    assert rows == p.S * (parts + probes)
    X, y = g.surrogate_dataset()
    pos_g, n_g, _, _ = g.get_walkers()
    o = O.Oracle(p, pos=pos_g, n=n_g, surrogate=theta_of(1))
    key = (int(p.seed) & 0xFFFFFFFF, int(p.seed) >> 32)
    checked = 0
    for w in range(p.S):
        N = int(n_g[w])
        for slot in range(parts + probes):
            r = w * (parts + probes) + slot
            if slot < parts and N > 0:
                i = slot * N // parts
                q = o.pos[w, i].copy()
                skip = i
            else:
                u = O.philox4x32_10([slot, w, 0, 5], key)
                q = np.array([np.float32(p.Lx) * np.float32((u[0] >> 8) / 16777216.0),
                              np.float32(p.Ly) * np.float32((u[1] >> 8) / 16777216.0),
                              np.float32(np.float32(p.z_lo) + np.float32(
                                  np.float32(p.z_hi - p.z_lo) * np.float32((u[2] >> 8) / 16777216.0)))],
                             np.float64)
                if q[0] >= np.float32(p.Lx):
                    q[0] = 0.0
                if q[1] >= np.float32(p.Ly):
                    q[1] = 0.0
                skip = -1
            _, fo = o.surrogate_energy(w, q, skip=skip)
            eo, sum_abs, band, _ = o.particle_energy(w, q, skip=skip)
            ws = weight_sum(p, np.delete(o.pos[w, :N], skip, axis=0) if skip >= 0 else o.pos[w], N - (skip >= 0), q)
            assert np.all(np.abs(X[r] - fo) <= feat_tol(fo, ws)), (w, slot, X[r] - fo)
            target = min(eo, clip)
            if eo > clip + 1e-4 * sum_abs + band:
                assert y[r] == np.float32(clip), (w, slot, y[r], eo)
            elif eo < clip - 1e-4 * sum_abs - band:
                assert abs(y[r] - target) <= 1e-5 * sum_abs + band + 1e-6, (w, slot, y[r], target)
            checked += 1
    assert checked == rows


def run_da_lockstep(p, pos, n, th, blocks, sweeps, exchange=True):
    g = Regc(p)
    g.set_walkers(pos, n)
    g.surrogate_set(th)
    g.set_mode(True)
    o = O.Oracle(p, pos=pos, n=n, surrogate=th)
    compared, exact, diverged = 0, 0, []
    screened = passed = 0
    for b in range(blocks):
        beta = 1.0 / np.asarray(p.kT)[o.state_of_walker // p.M]
        tg = g.sweep_traced(sweeps)
        to = o.sweeps(sweeps, trace=True)
        c, x, d = compare_da_traces(tg, to, beta, sur_tol_of)
        compared += c
        exact += x
        ev = to["status"] == 0
        screened += int(ev.sum())
        passed += int((to["stage1"][ev] == 1).sum())
        if d:
            diverged = d
            break
        if exchange:
            g.exchange()
            o.exchange()
    return g, o, compared, exact, diverged, screened, passed


def assert_same_final_state(g, o, p, screened, passed):
    pos, n, e, sow = g.get_walkers()
    assert np.array_equal(n, o.n)
    assert np.array_equal(sow, o.state_of_walker)
    for w in range(p.S):
        assert np.array_equal(pos[w, :n[w]], o.pos[w, :n[w]].astype(np.float32)), "walker %d" % w
    assert np.all(np.abs(e - o.energy) <= 1e-4 * np.maximum(1.0, np.abs(o.energy)))
    mv, ex, pr = g.counters()
    assert np.array_equal(mv, o.counts)
    assert np.array_equal(ex, o.ex_counts)
    assert pr[4] == screened and pr[5] == passed
    assert g.check_energy() == 0.0


def test_da_lockstep_fcc100_16_replicas():
    p = W.fcc100_small()
    rng = np.random.default_rng(0)
    pos, n = W.initial_walkers(p, rng.integers(0, 25, p.S), seed=1)
    g, o, compared, exact, diverged, screened, passed = run_da_lockstep(p, pos, n, theta_of(2), blocks=8,
                                                                        sweeps=10)
    assert compared >= p.S * 20 * 10
    assert 0 < passed < screened, (passed, screened)   # the screen decided some moves
    if not diverged:
        assert_same_final_state(g, o, p, screened, passed)


@pytest.mark.parametrize("case", ["empty_walkers", "ragged_nmax_37_full", "displacement_only", "gc_only",
                                  "dense_slab_long_columns",
                                  "moves_45_p_disp_08", "periodic_cube_no_surface", "one_cell_per_axis"])
def test_da_lockstep_edge_cases(case):
    p, n0 = EDGE_CASES[case]()
    if n0 == "full":
        n0 = p.nmax
    elif n0 == "half":
        n0 = np.arange(p.S) % 2
    pos, n = W.initial_walkers(p, n0, seed=7, min_dist=0.85)
    g, o, compared, exact, diverged, screened, passed = run_da_lockstep(p, pos, n, theta_of(3, 0.8),
                                                                        blocks=4, sweeps=5)
    if not diverged:
        assert_same_final_state(g, o, p, screened, passed)


def test_da_production_kernel_matches_traced_kernel():
    p = W.fcc100_small()
    pos, n = W.initial_walkers(p, 15, seed=4)
    runs = []
    for traced in (False, True):
        g = Regc(p)
        g.set_walkers(pos, n)
        g.surrogate_set(theta_of(5))
        g.set_mode(True)
        for _ in range(3):
            if traced:
                g.sweep_traced(10)
            else:
                g.sweep(10)
            g.exchange()
        runs.append(g.get_walkers())
    for x, y in zip(*runs):
        assert np.array_equal(x, y)


def trunc_poisson(lam, nmax):
    k = np.arange(nmax + 1)
    lp = k * math.log(lam) - np.array([math.lgamma(i + 1) for i in k])
    q = np.exp(lp - lp.max())
    return q / q.sum()


def test_da_ideal_gas_truncated_poisson_untrained_network():
    p = W.ideal_gas(W.fcc100_small()).replace(moves_per_sweep=3, p_disp=0.0)
    th = theta_of(9, 1.5)
    th[-1] = 0.7    # e~ is a constant 0.7 + ... at G = 0: a biased screen
    g = Regc(p)
    g.surrogate_set(th)
    g.set_mode(True)
    g.run(200, exchange_every=1)
    g.reset_histograms()
    nb = []
    nv = np.arange(p.nmax + 1)
    prev = g.histograms()["hN"]
    for b in range(16):
        g.run(2000, exchange_every=1)
        h = g.histograms()["hN"]
        d = h - prev
        prev = h
        nb.append((d @ nv) / d.sum(axis=1))
    nb = np.array(nb)
    V = p.Lx * p.Ly * (p.z_hi - p.z_lo)
    for s in range(p.S):
        kT, mu = p.kT[s // p.M], p.mu[s % p.M]
        lam = V * math.exp(mu / kT) / (p.lambda0 / math.sqrt(kT)) ** 3
        exp_mean = trunc_poisson(lam, p.nmax) @ nv
        se = nb[:, s].std(ddof=1) / math.sqrt(len(nb))
        assert abs(nb[:, s].mean() - exp_mean) <= 4.5 * se + 1e-3, (s, nb[:, s].mean(), exp_mean, se)


def sample_counts(g, sweeps):
    g.reset_histograms()
    g.run(sweeps, exchange_every=10)
    mv, ex, pr = g.counters()
    h = g.histograms()
    return mv, pr, h


def test_training_lowers_loss_and_trained_network_screens():
    p = W.fcc100_small()
    rng = np.random.default_rng(2)
    pos, n = W.initial_walkers(p, rng.integers(0, 20, p.S), seed=2)
    g = Regc(p)
    g.set_walkers(pos, n)
    th0 = SG.init_params(11, scale=1.0).astype(np.float32)
    g.surrogate_set(th0)
    g.run(200, exchange_every=10)
    for _ in range(100):
        g.run(10, exchange_every=10)
        rows = g.surrogate_harvest(8, 8, 8.0, capacity=100 * p.S * 16)
    assert rows == 100 * p.S * 16
    loss = g.surrogate_train(1500, 512, 2e-3)
    first, last = float(np.mean(loss[:20])), float(np.mean(loss[-100:]))
    print("training loss %.4g -> %.4g" % (first, last))
    assert last < 0.25 * first
    state = g.get_walkers()

    def measure(theta, delayed):
        h = Regc(p)
        h.set_walkers(state[0], state[1], state[3])
        if theta is not None:
            h.surrogate_set(theta)
        h.set_mode(delayed)
        h.run(100, exchange_every=10)
        return sample_counts(h, 1000)

    trained = g.surrogate_get()
    mv_p, pr_p, h_p = measure(None, False)
    mv_t, pr_t, h_t = measure(trained, True)
    mv_u, pr_u, h_u = measure(th0, True)
    acc = lambda mv: mv[:, :, 1].sum()           # noqa: E731
    trials = lambda mv: mv[:, :, 0].sum()        # noqa: E731
    # exact energy evaluations per accepted move: every evaluated move for the
    # plain sweep; only the moves that passed the screen with delayed acceptance
    ev_plain = pr_p[3] / acc(mv_p)
    ev_trained = pr_t[5] / acc(mv_t)
    ev_untrained = pr_u[5] / acc(mv_u)
    print("exact evaluations per accepted move: plain %.3g, trained %.3g, untrained %.3g"
          % (ev_plain, ev_trained, ev_untrained))
    print("acceptance: plain %.4g, trained %.4g, untrained %.4g"
          % (acc(mv_p) / trials(mv_p), acc(mv_t) / trials(mv_t), acc(mv_u) / trials(mv_u)))
    assert ev_trained < 0.5 * ev_plain
    assert ev_trained < ev_untrained
    # the trained screen passes moves the exact stage then accepts
    assert acc(mv_t) / pr_t[5] > acc(mv_u) / max(pr_u[5], 1)


def test_seeded_initial_parameters():
    p = W.fcc100_small(L=1, M=1)
    g = Regc(p)
    g.surrogate_init(seed=3, scale=1.0)
    a = g.surrogate_get()
    g.surrogate_init(seed=3, scale=1.0)
    assert np.array_equal(a, g.surrogate_get())
    g.surrogate_init(seed=4, scale=2.0)
    b = g.surrogate_get()
    m = SG.weight_mask()
    assert np.all(a[~m] == 0.0) and np.all(b[~m] == 0.0)
    W1, _, W2, _, W3, _ = SG.unpack(a)
    for w, fan in ((W1, 16), (W2, 64), (W3, 64)):
        z = np.ravel(w) * math.sqrt(fan)
        # mean 0 and variance 1 within 5 standard errors
        assert abs(z.mean()) < 5 / math.sqrt(z.size)
        assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    z = np.ravel(SG.unpack(b)[2]) * 8.0 / 2.0
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert not np.array_equal(np.ravel(SG.unpack(b)[2]) / 2.0, np.ravel(W2))
