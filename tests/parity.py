"""Move-by-move comparison of a GPU trace with an oracle trace.

Both implementations start from the same configurations and draw the same
Philox numbers, and their coordinate arithmetic is the same binary32
arithmetic, so they make identical moves for as long as their accept/reject
decisions agree.  The GPU's pair energies are binary32 and the oracle's FP64,
so a decision may differ only when the oracle's ln u lies within the energy
tolerance of its log acceptance ratio (a near-tie); after such a divergence
the two chains are no longer comparable for that walker.

Energy tolerance (per move): |dE_gpu - dE_oracle| <= 1e-5 max(|dE|, T), where
T = sum over the pairs entering dE of 4 eps [(sigma/r)^12 + (sigma/r)^6] (the
two terms of the LJ pair energy cancel near r = sigma, so |phi| alone would
understate the binary32 rounding), plus the step of phi at rc for every pair
within 4e-6 rc^2 of the cutoff, plus half a unit of the GPU's fixed-point
energy grid (2^-30) per pair within rc.
"""
import numpy as np

DE_REL = 1e-5


def de_tolerance(o):
    # + half a fixed-point unit (2^-30) per pair: the GPU rounds every pair
    # energy onto that grid before summing (visible when energies are small in
    # the problem's units, e.g. eV for weak gas-gas pairs)
    return DE_REL * np.maximum(np.abs(o["dE"]), o["sum_abs"]) + o["band"] + o["n_pairs"] * 2.0 ** -31 + 1e-9


def compare_traces(gt, ot, beta_max):
    """Compare [S, ...] traces walker by walker.

    Returns (n_moves_compared, diverged_walkers).  Raises AssertionError on any
    disagreement that is not explained by a near-tie."""
    S = gt.shape[0]
    g = gt.reshape(S, -1)
    o = ot.reshape(S, -1)
    compared = 0
    diverged = []
    for w in range(S):
        for k in range(g.shape[1]):
            a, b = g[w, k], o[w, k]
            where = "walker %d move %d" % (w, k)
            assert a["type"] == b["type"], where + ": move type"
            assert a["status"] == b["status"], where + ": status %d vs %d" % (a["status"], b["status"])
            assert a["index"] == b["index"], where + ": index"
            assert abs(a["ln_u"] - b["ln_u"]) < 1e-12, where + ": ln u"
            tol = 0.0
            if b["status"] == 0:
                if b["dE"] > 1e5:
                    # a pair inside the hard-core guard: both sides must reject
                    assert not a["accepted"] and not b["accepted"], where + ": overlap accepted"
                else:
                    tol = de_tolerance(b)
                    assert abs(a["dE"] - b["dE"]) <= tol, \
                        where + ": dE %.9g vs %.9g (tol %.3g)" % (a["dE"], b["dE"], tol)
                    if b["band"] == 0.0:
                        assert a["n_pairs"] == b["n_pairs"], where + ": pairs in range"
            compared += 1
            if a["accepted"] != b["accepted"]:
                margin = abs(b["ln_u"] - b["log_alpha"])
                assert margin <= beta_max * tol + 1e-6, \
                    where + ": decisions differ outside the near-tie band (margin %.3g)" % margin
                diverged.append(w)
                break
    return compared, diverged


def compare_da_traces(gt, ot, beta, sur_tol):
    """Compare delayed-acceptance traces walker by walker.

    beta [S]: inverse temperature of each walker's state during the traced
    sweeps.  sur_tol(o) -> tolerance of the surrogate energy change dE~ of each
    oracle record (binary32 features and activations against FP64).

    Stage 1 (ln u1 < la + beta (dE - dE~), la the plain log ratio) may differ
    only where ln u1 lies within beta * sur_tol of its threshold; stage 2
    (ln u < -beta (dE - dE~)) only within beta * (dE tol + sur_tol).  After a
    differing decision the walker is no longer compared.

    Returns (n_moves_compared, n_exact_evaluations_compared, diverged_walkers)."""
    S = gt.shape[0]
    g = gt.reshape(S, -1)
    o = ot.reshape(S, -1)
    compared, exact, diverged = 0, 0, []
    for w in range(S):
        bw = float(beta[w])
        for k in range(g.shape[1]):
            a, b = g[w, k], o[w, k]
            where = "walker %d move %d" % (w, k)
            assert a["type"] == b["type"], where + ": move type"
            assert a["status"] == b["status"], where + ": status %d vs %d" % (a["status"], b["status"])
            assert a["index"] == b["index"], where + ": index"
            assert abs(a["ln_u"] - b["ln_u"]) < 1e-12, where + ": ln u"
            compared += 1
            if b["status"] != 0:
                assert not a["accepted"] and not b["accepted"], where + ": status move accepted"
                continue
            assert abs(a["ln_u1"] - b["ln_u1"]) < 1e-12, where + ": ln u1"
            ts = float(sur_tol(b))
            assert abs(a["dE_sur"] - b["dE_sur"]) <= ts, \
                where + ": dE~ %.9g vs %.9g (tol %.3g)" % (a["dE_sur"], b["dE_sur"], ts)
            hard = b["dE"] > 1e5
            if a["stage1"] != b["stage1"]:
                # la1 = c - beta dE~ with c = la + beta dE (not rebuilt for an overlap,
                # where la has lost c's digits: a differing screen there fails)
                assert not hard, where + ": stage-1 decisions differ on an overlapping move"
                la1 = b["log_alpha"] + bw * (b["dE"] - b["dE_sur"])
                margin = abs(b["ln_u1"] - la1)
                assert margin <= bw * ts + 1e-6, \
                    where + ": stage-1 decisions differ outside the near-tie band (margin %.3g)" % margin
                diverged.append(w)
                break
            if not b["stage1"]:
                assert np.isnan(a["dE"]), where + ": dE evaluated after a stage-1 rejection"
                assert not a["accepted"] and not b["accepted"], where + ": screened move accepted"
                continue
            exact += 1
            tol = 0.0
            if hard:
                assert not a["accepted"] and not b["accepted"], where + ": overlap accepted"
            else:
                tol = de_tolerance(b)
                assert abs(a["dE"] - b["dE"]) <= tol, \
                    where + ": dE %.9g vs %.9g (tol %.3g)" % (a["dE"], b["dE"], tol)
            if a["accepted"] != b["accepted"]:
                la2 = -bw * (b["dE"] - b["dE_sur"])
                margin = abs(b["ln_u"] - la2)
                assert margin <= bw * (tol + ts) + 1e-6, \
                    where + ": stage-2 decisions differ outside the near-tie band (margin %.3g)" % margin
                diverged.append(w)
                break
    return compared, exact, diverged
