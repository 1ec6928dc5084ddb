"""Pins of the oracle's molecular-dynamics step (REGCMD: Sec. II.A.3 with MD as
the canonical sampler; Appendix: velocity Verlet and the stochastic velocity
rescaling thermostat).

* Forces are minus the gradient of the oracle's energy (central finite
  differences), for gas particles near the surface and for cluster atoms.
* The thermostat (Bussi, Donadio & Parrinello 2007) keeps the kinetic energy
  of an ideal gas distributed as Gamma(3N/2, kT): mean 3N kT / 2 and variance
  3N kT^2 / 2 after many thermostat steps; dropping the cross term of the
  rescaled kinetic energy (planted) is detected.
* MD alone samples the canonical ensemble: one particle above the small box's
  surface has the brute-force mean energy at every temperature (the time step
  is small enough for its bias to stay below the statistical error); forces
  of the wrong sign (planted) are detected.
* Grand-canonical moves alternated with MD segments (REGCMD) reproduce the
  brute-force <N> and <E> of the small box.
* Velocity Verlet conserves the total energy over short segments of a dilute
  system without the thermostat.
* The REGCMD cycle (the x0 choice of Sec. II.A, then an MD segment) keeps the
  small box's brute-force <N> and <E>; a dropped 1/(N+1) and wrong-sign
  forces (planted) are caught.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from test_oracle_pins import brute_force_small_box, small_box_problem


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def test_forces_are_minus_the_energy_gradient():
    for p, pos, n in (
        (W.fcc100_small(L=1, M=1, seed=2),) + tuple(W.initial_walkers(W.fcc100_small(L=1, M=1), 12, seed=5)),
        (W.cluster_in_gas(L=1, M=1, nmax_b=12, box=6.0),) + tuple(W.cluster_initial(
            W.cluster_in_gas(L=1, M=1, nmax_b=12, box=6.0), 8, seed=3)),
    ):
        o = O.Oracle(p, pos=pos, n=n)
        f = o.forces(0)
        h = 1e-6
        for i in range(int(n[0])):
            for c in range(3):
                save = o.pos[0, i, c]
                o.pos[0, i, c] = save + h
                ep = o.total_energy(0)
                o.pos[0, i, c] = save - h
                em = o.total_energy(0)
                o.pos[0, i, c] = save
                fd = -(ep - em) / (2 * h)
                assert abs(fd - f[i, c]) <= 1e-5 * max(1.0, abs(f[i, c])), (i, c, fd, f[i, c])


def kinetic_pin(mutation=0, segments=400):
    p = W.ideal_gas(W.fcc100_small(L=1, M=2, seed=4))
    pos, n = W.initial_walkers(p, 10, seed=6)
    o = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    ks = np.array([o.md(40, 0.01, 0.05) for _ in range(segments)])     # [segments, S]
    worst = 0.0
    for w in range(p.S):
        kT = p.kT[o.state_of_walker[w] // p.M]
        nf = 3 * int(n[w])
        mean, var = nf * kT / 2, nf * kT * kT / 2
        k = ks[:, w]
        z_mean = (k.mean() - mean) / math.sqrt(var / len(k))
        # variance of the sample variance of a Gamma(a, kT): kT^4 (2 a^2 + 6 a) / n with a = nf / 2
        a = nf / 2
        z_var = (k.var(ddof=1) - var) / math.sqrt(kT ** 4 * (2 * a * a + 6 * a) / len(k))
        worst = max(worst, abs(z_mean), abs(z_var))
    return worst


def test_thermostat_keeps_the_canonical_kinetic_energy():
    assert kinetic_pin() < 4.5


def test_planted_thermostat_mistake_is_detected():
    assert kinetic_pin(mutation=512) > 6.0


def regcmd_small_box(mutation=0, cycles=6000):
    """<N>, <E> of the small box with GC-only sweeps and MD segments."""
    p = small_box_problem().replace(p_disp=0.0, moves_per_sweep=4)
    o = O.Oracle(p, mutation=mutation)
    nb, eb = [], []
    nv = np.arange(p.nmax + 1)
    for b in range(16):
        h0, m0, om0 = o.hN.copy(), o.moments.copy(), o.omega.copy()
        for c in range(cycles // 16):
            o.sweeps(1)
            o.md(10, 0.005, 0.1)
            if c % 10 == 9:
                o.exchange()
        dh = o.hN - h0
        nb.append((dh @ nv) / np.maximum(dh.sum(axis=1), 1))
        eb.append((o.moments[:, 2] - m0[:, 2]) / np.maximum(o.omega - om0, 1))
    return p, np.array(nb), np.array(eb)


def expected_small_box(p):
    bf = brute_force_small_box(p)
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
    return exp_n, exp_e, sd_n


@pytest.mark.slow
def test_regcmd_small_box_brute_force():
    p, nb, eb = regcmd_small_box()
    exp_n, exp_e, sd_n = expected_small_box(p)
    zn = (nb.mean(axis=0) - exp_n) / (nb.std(axis=0, ddof=1) / 4.0)
    ze = (eb.mean(axis=0) - exp_e) / (eb.std(axis=0, ddof=1) / 4.0)
    assert max(np.max(np.abs(zn)), np.max(np.abs(ze))) < 4.5, (zn, ze)


def canonical_one_particle(mutation=0, segments=3000):
    """MD alone (fixed N = 1): mean potential energy of one particle above the
    small box's surface per temperature, from the end of each segment."""
    p = small_box_problem()
    pos = np.zeros((p.S, p.nmax, 3))
    pos[:, 0] = [1.3, 1.3, 2.0]
    n = np.ones(p.S, np.int32)
    o = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    es = []
    for k in range(segments):
        o.md(25, 0.005, 0.05)
        es.append(o.energy.copy())
    es = np.array(es)[segments // 10:]
    nb = 20
    b = es[: len(es) // nb * nb].reshape(nb, -1, p.S).mean(axis=1)
    bf = brute_force_small_box(p)
    z = []
    for s in range(p.S):
        e1 = bf[float(p.kT[s // p.M])][2]
        z.append((b[:, s].mean() - e1) / (b[:, s].std(ddof=1) / math.sqrt(nb)))
    return float(np.max(np.abs(z)))


def test_md_samples_the_canonical_energy_of_one_particle():
    assert canonical_one_particle() < 4.5


def test_planted_force_sign_mistake_is_detected():
    assert canonical_one_particle(mutation=1024, segments=800) > 6.0


def test_velocity_verlet_conserves_energy_without_thermostat():
    # dilute LJ gas in a periodic cube, thermostat off (tau huge): E + K drifts
    # only by the jumps of the truncated potential at rc, none here at low density
    p = W.Problem(n_types=1, eps=np.diag([1.0, 0, 0, 0]), sigma=np.ones((4, 4)), rc=2.5, Lx=8.0, Ly=8.0, Lz=8.0,
                  periodic_z=1, z_lo=0.0, z_hi=8.0, surf_xyz=np.zeros((0, 3)), surf_type=np.zeros(0, np.int32),
                  kT=np.array([1.0]), mu=np.array([-3.0]), lambda0=1.0, nmax=8, moves_per_sweep=1,
                  max_disp=0.1, p_disp=0.5, seed=1, e_lo=-50.0, e_bin=0.1, n_e_bins=1000)
    pos = np.zeros((1, 8, 3))
    pos[0, :2] = [[2.0, 2.0, 2.0], [3.2, 2.1, 2.0]]     # one bound-ish pair well inside rc
    n = np.array([2], np.int32)
    a = O.Oracle(p, pos=pos, n=n)
    b = O.Oracle(p, pos=pos, n=n)
    k0 = a.md(0, 0.001, 1e12)[0]          # the same starting velocities (segment 0), no steps
    k1 = b.md(400, 0.001, 1e12)[0]
    d = (b.energy[0] + k1) - (a.energy[0] + k0)
    assert abs(d) < 2e-3 * max(1.0, abs(a.energy[0] + k0)), d


def regcmd_cycle_small_box(mutation=0, steps=6000, x0=0.9):
    """<N>, <E> of the small box under the REGCMD cycle: per step the x0
    choice (particle exchange or replica exchange), then one MD segment."""
    p = small_box_problem().replace(p_disp=0.0)
    o = O.Oracle(p, mutation=mutation)
    nb, eb = [], []
    nv = np.arange(p.nmax + 1)
    for b in range(16):
        h0, m0, om0 = o.hN.copy(), o.moments.copy(), o.omega.copy()
        o.cycle_md(steps // 16, x0, 10, 0.005, 0.1)
        dh = o.hN - h0
        nb.append((dh @ nv) / np.maximum(dh.sum(axis=1), 1))
        eb.append((o.moments[:, 2] - m0[:, 2]) / np.maximum(o.omega - om0, 1))
    return p, np.array(nb), np.array(eb)


def test_regcmd_cycle_small_box_brute_force():
    p, nb, eb = regcmd_cycle_small_box()
    exp_n, exp_e, sd_n = expected_small_box(p)
    zn = (nb.mean(axis=0) - exp_n) / (nb.std(axis=0, ddof=1) / 4.0)
    ze = (eb.mean(axis=0) - exp_e) / (eb.std(axis=0, ddof=1) / 4.0)
    assert max(np.max(np.abs(zn)), np.max(np.abs(ze))) < 4.5, (zn, ze)


@pytest.mark.parametrize("bit", [8, 1024])
def test_planted_mistakes_under_the_regcmd_cycle(bit):
    """The dropped 1/(N+1) of the insertion rule (8) and wrong-sign forces
    (1024) both break the small-box pin under the REGCMD cycle (the latter
    drives particles together until the energies are no longer finite)."""
    p, nb, eb = regcmd_cycle_small_box(mutation=bit)
    exp_n, exp_e, sd_n = expected_small_box(p)
    zn = (nb.mean(axis=0) - exp_n) / (nb.std(axis=0, ddof=1) / 4.0)
    ze = (eb.mean(axis=0) - exp_e) / (eb.std(axis=0, ddof=1) / 4.0)
    worst = np.max(np.abs(np.concatenate([zn, ze])))        # NaN (non-finite energies) counts as caught
    assert not worst < 6.0, worst
