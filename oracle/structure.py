"""FP64 oracle of the structural observables of Sec. III.A ("Structural
properties") and of their MBAR averages per phase (Sec. II.B, Eq. avegr).

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU baseline,
never by the library.

Per sample (one walker's configuration, grand-canonical species only):

* axial distribution: particles counted in slabs of width dz parallel to the
  surface, slab k of a particle at height z being floor((z - z_lo) * (1/dz));
* lateral RDF of a layer l (particles with layer_lo[l] <= z < layer_hi[l]):
  unordered pairs of the layer counted by their distance in the xy plane
  (nearest image in x and y), bin k = floor(r * (1/dr)).

Like every geometric input of the C ABI, coordinates, z_lo, the periods, the
shear, dz and dr are binary32 values.  The bins are decided from them in
FP64 (the paper fixes no precision): slab k = floor((z - z_lo) / dz); the
lateral distance r = sqrt(dx^2 + dy^2) with du, dy the nearest-image
differences along the cell's axes and, in a sheared cell (cell-frame x), the
Cartesian dx = du + shear dy; bin k = floor(r / dr).  An implementation that
takes these decisions in binary32 can land on the other side of an edge only
for a value within a few binary32 roundings of it: ``sample_counts`` lists
every count whose value (in units of its bin width) lies within EDGE_REL of
an edge, with the bin on the other side.  Everything after the counts is
FP64.

Per configuration the functions of Sec. III.A are
  rho(z_k) = c_k / (A dz)                                (number density)
  g_xy(r_k) = 2 A P_k / (M (M - 1) pi (r_{k+1}^2 - r_k^2))   (M >= 2, else 0)
with A = Lx Ly, c_k the slab count, P_k the pair count of the layer and M its
population (the normalisation that gives g_xy = 1 for uniformly placed points).

MBAR average per phase (Eq. avegr, the phase i being N_B = i): every sample
is a bin of its own, (N_n, E_n), count 1; the MBAR free energies of the
sampled states follow from the solve of oracle/mbar.py, and the weight of
sample n at the query state q is
  W_n(q) = exp(-u_q(N_n, E_n) - D_n + f_q),  sum over all n of W_n(q) = 1.
Eq. avegr as printed sums W_n(q) g(r; R_n) over the samples of phase i, the
joint average of [N = i] g.  The average of g within phase i divides that by
p_i(q) = sum over the samples of phase i of W_n(q); both are returned.
"""
from __future__ import annotations

import math

import numpy as np

from . import mbar as MB

F = np.float32

# relative distance to a bin edge within which a binary32 decision (a handful
# of roundings of 2^-24 each) may differ from the FP64 one
EDGE_REL = 1e-6


def _bin_of(v, edges, kind, layer):
    """floor(v), and the neighbouring bin if v lies within EDGE_REL of an edge
    (appended to edges as (kind, layer, k, k_other))."""
    k = math.floor(v)
    tol = EDGE_REL * max(1.0, abs(v))
    if edges is not None:
        if v - k < tol:
            edges.append((kind, layer, k, k - 1))
        elif k + 1 - v < tol:
            edges.append((kind, layer, k, k + 1))
    return k


def _min_image(d, L):
    """Nearest-image difference along a periodic axis of period L (FP64)."""
    if d > 0.5 * L:
        return d - L
    if d < -0.5 * L:
        return d + L
    return d


def sample_counts(problem, pos_w, n_w, spec, mutation: int = 0, edges=None):
    """Counts of one configuration: (slab counts [n_z], pair counts
    [n_layers, n_r], layer populations [n_layers]).

    spec: dict with n_z, dz, layers [(lo, hi), ...], n_r, dr.
    edges: a list that receives (kind 'rho' or 'pairs', layer, k, k_other) for
    every count whose bin decision lies within EDGE_REL of an edge (bins out
    of range included, so a count may appear or vanish).
    mutation 1: slab index one too high; 2: ordered pairs counted twice."""
    n_z, n_r = int(spec["n_z"]), int(spec["n_r"])
    layers = list(spec["layers"])
    dz, dr = float(F(spec["dz"])), float(F(spec["dr"]))
    z_lo = float(F(problem.z_lo))
    Lx, Ly = float(F(problem.Lx)), float(F(problem.Ly))
    shear = float(F(getattr(problem, "shear", 0.0)))
    first = int(getattr(problem, "n_cluster", 0))
    pts = [tuple(float(F(c)) for c in pos_w[j]) for j in range(first, int(n_w))]
    rho = np.zeros(n_z, np.int64)
    for (_, _, z) in pts:
        k = _bin_of((z - z_lo) / dz, edges, "rho", -1)
        if mutation & 1:
            k += 1
        if 0 <= k < n_z:
            rho[k] += 1
    pairs = np.zeros((len(layers), n_r), np.int64)
    pop = np.zeros(len(layers), np.int64)
    for l, (lo, hi) in enumerate(layers):
        lo, hi = float(F(lo)), float(F(hi))
        mem = [q for q in pts if lo <= q[2] < hi]
        pop[l] = len(mem)
        for a in range(len(mem)):
            for b in range(a + 1, len(mem)):
                dy = _min_image(mem[a][1] - mem[b][1], Ly)
                dx = _min_image(mem[a][0] - mem[b][0], Lx) + shear * dy
                k = _bin_of(math.sqrt(dx * dx + dy * dy) / dr, edges, "pairs", l)
                if k < n_r:
                    pairs[l, k] += 2 if mutation & 2 else 1
    return rho, pairs, pop


def structure_of_walkers(problem, pos, n, state_of_walker, energy, spec, edges=None):
    """One sample per walker: dict of arrays state [S], N [S] (grand-canonical
    count), E [S], rho [S, n_z], pairs [S, n_layers, n_r], pop [S, n_layers].
    edges: a list that receives one list per walker (see sample_counts)."""
    S = len(n)
    first = int(getattr(problem, "n_cluster", 0))
    out = {"state": np.array(state_of_walker, np.int64), "N": np.array(n, np.int64) - first,
           "E": np.array(energy, np.float64),
           "rho": np.zeros((S, spec["n_z"]), np.int64),
           "pairs": np.zeros((S, len(spec["layers"]), spec["n_r"]), np.int64),
           "pop": np.zeros((S, len(spec["layers"])), np.int64)}
    for w in range(S):
        ew = [] if edges is not None else None
        r, p, m = sample_counts(problem, pos[w], n[w], spec, edges=ew)
        out["rho"][w], out["pairs"][w], out["pop"][w] = r, p, m
        if edges is not None:
            edges.append(ew)
    return out


def edge_moves(counts, reference, edges):
    """Reconcile another implementation's counts with the oracle's.

    counts, reference: dicts with rho [n, n_z] and pairs [n, n_layers, n_r]
    (the other implementation's, the oracle's); edges: per sample the list
    from sample_counts.  A count may differ from the oracle's only by a
    near-edge item that landed in the neighbouring bin.  Returns (unexplained,
    moved): the counts that no such move explains, and the items moved."""
    bad = moved = 0
    n_layers = reference["pairs"].shape[1]
    for w in range(reference["rho"].shape[0]):
        res = {("rho", -1): np.asarray(counts["rho"][w], np.int64) - reference["rho"][w]}
        for l in range(n_layers):
            res[("pairs", l)] = np.asarray(counts["pairs"][w, l], np.int64) - reference["pairs"][w, l]
        for kind, l, k, k2 in edges[w]:
            r = res[(kind, l)]
            src, dst = 0 <= k < len(r), 0 <= k2 < len(r)
            if (src or dst) and (not src or r[k] < 0) and (not dst or r[k2] > 0):
                if src:
                    r[k] += 1
                if dst:
                    r[k2] -= 1
                moved += 1
        bad += sum(int(np.abs(r).sum()) for r in res.values())
    return bad, moved


def concat(samples):
    return {k: np.concatenate([s[k] for s in samples]) for k in samples[0]}


def concat_edges(edge_lists):
    """Concatenate the per-sample edge lists of several structure_of_walkers calls."""
    return [e for lst in edge_lists for e in lst]


def reweight(problem, samples, spec, kT_q, mu_q, n_lo, n_hi, tol=1e-10, max_iter=200000, mutation: int = 0):
    """MBAR averages per phase N_B = n_lo..n_hi at the query states.

    Returns dict: f [S] (sampled states, f_0 = 0), p [Q, phases] (probability
    of each phase), rho [Q, phases, n_z] and gxy [Q, phases, n_layers, n_r]
    (averages within each phase; zero where p = 0), joint_rho and joint_gxy
    (Eq. avegr as printed: the same sums without the division by p).
    mutation 4: the 3 N ln Lambda term left out of the query's reduced potential."""
    kT_s = np.asarray(problem.kT)[np.arange(problem.S) // problem.M]
    mu_s = np.asarray(problem.mu)[np.arange(problem.S) % problem.M]
    st, N, E = samples["state"], samples["N"].astype(np.float64), samples["E"]
    omega = np.bincount(st, minlength=problem.S).astype(np.float64)
    lam0 = problem.lambda0
    f, D, _, _ = MB.solve(kT_s, mu_s, lam0, omega, N, E, np.ones(len(N)), tol=tol, max_iter=max_iter)
    u = MB.reduced_potential(kT_q, mu_q, lam0, N, E)             # [Q, n]
    if mutation & 4:
        kq = np.atleast_1d(np.asarray(kT_q, np.float64))[:, None]
        u = u - 3.0 * N[None, :] * (math.log(lam0) - 0.5 * np.log(kq))
    ln_w = -u - D[None, :]
    f_q = -MB.lse(ln_w, axis=1)
    W = np.exp(ln_w + f_q[:, None])                                # [Q, n], rows sum to 1
    A = problem.Lx * problem.Ly
    dz, dr = float(F(spec["dz"])), float(F(spec["dr"]))
    n_r = int(spec["n_r"])
    shell = math.pi * dr * dr * ((np.arange(n_r) + 1.0) ** 2 - np.arange(n_r) ** 2)
    pop = samples["pop"].astype(np.float64)
    norm = np.where(pop >= 2, 2.0 * A / np.maximum(pop * (pop - 1.0), 1.0), 0.0)       # [n, layers]
    g_n = samples["pairs"] * norm[:, :, None] / shell[None, None, :]                      # [n, layers, n_r]
    rho_n = samples["rho"] / (A * dz)                                                     # [n, n_z]
    Q, P = W.shape[0], n_hi - n_lo + 1
    out = {"f": f, "p": np.zeros((Q, P)), "rho": np.zeros((Q, P, rho_n.shape[1])),
           "gxy": np.zeros((Q, P) + g_n.shape[1:]), "joint_rho": np.zeros((Q, P, rho_n.shape[1])),
           "joint_gxy": np.zeros((Q, P) + g_n.shape[1:])}
    for i in range(P):
        sel = samples["N"] == n_lo + i
        if not np.any(sel):
            continue
        w = W[:, sel]
        out["p"][:, i] = w.sum(axis=1)
        out["joint_rho"][:, i] = w @ rho_n[sel]
        out["joint_gxy"][:, i] = np.tensordot(w, g_n[sel], axes=(1, 0))
        ok = out["p"][:, i] > 0
        out["rho"][ok, i] = out["joint_rho"][ok, i] / out["p"][ok, i][:, None]
        out["gxy"][ok, i] = out["joint_gxy"][ok, i] / out["p"][ok, i][:, None, None]
    return out
