"""Pins of the oracle in a sheared cell (the paper's own cell for the LJ
surface of Sec. III.A: the 3 x 3 hexagonal supercell of fcc(111), lattice
vectors of 11.489 A at 60 degrees; coordinates in the cell frame u = x - y
tan 30).

* Energies against a plain numpy sum over the Cartesian image lattice.
* The same physical configuration described in the hexagonal cell and,
  doubled, in the rectangular cell that holds two of them: the rectangular
  energy is twice the hexagonal one.
* MD forces are minus the gradient of the energy with respect to the
  Cartesian coordinates (finite differences through the cell frame).
* One particle above the slab sampled by Metropolis displacements in the cell
  frame: its canonical mean energy equals the quadrature over the cell.
* Leaving the nearest-image search along y out (planted) breaks the first pin.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def lj(r2, eps, sig, rc):
    s6 = (sig * sig / r2) ** 3
    return np.where(r2 < rc * rc, 4.0 * eps * (s6 * s6 - s6), 0.0)


def lattice_energy(p, pos, n):
    """E of one configuration: every mobile-mobile pair and mobile-surface
    pair over the images i A1 + j A2, |i|, |j| <= 2, in Cartesian coordinates."""
    A1 = np.array([p.Lx, 0.0, 0.0])
    A2 = np.array([p.shear * p.Ly, p.Ly, 0.0])
    shifts = np.array([i * A1 + j * A2 for i in range(-2, 3) for j in range(-2, 3)])
    C = W.cartesian(p, pos[:n])
    Sx = W.cartesian(p, p.surf_xyz)
    e = 0.0
    for i in range(n):
        d = C[i][None, None, :] - Sx[None, :, :] + shifts[:, None, :]
        e += lj(np.sum(d * d, axis=2), p.eps[0, 1], p.sigma[0, 1], p.rc).sum()
        for j in range(i + 1, n):
            d = C[i] - C[j] + shifts
            e += lj(np.sum(d * d, axis=1), p.eps[0, 0], p.sigma[0, 0], p.rc).sum()
    return e


def hex_walkers(p, n_b, seed):
    return W.lj_a18_initial(p, n_b, seed=seed)


def energy_pin(mutation=0):
    p = W.lj_a18_hex_slab(L=2, M=2, nmax=64, seed=1)
    pos, n = hex_walkers(p, [0, 12, 30, 50], seed=2)
    o = O.Oracle(p, pos=pos, n=n, mutation=mutation)
    worst = 0.0
    for w in range(p.S):
        ref = lattice_energy(p, pos[w], n[w])
        worst = max(worst, abs(o.total_energy(w) - ref) / max(1.0, abs(ref)))
    return worst


def test_energies_match_the_image_lattice_sum():
    assert energy_pin() < 1e-12


def test_planted_missing_y_image_is_detected():
    assert energy_pin(mutation=32) > 1e-6


def test_hexagonal_cell_equals_half_the_rectangular_cell():
    hexp = W.lj_a18_hex_slab(L=1, M=1, nmax=64, seed=3)
    rect = W.lj_a18_slab(L=1, M=1, nmax=128, seed=3)
    assert abs(rect.Lx - hexp.Lx) < 1e-5 and abs(rect.Ly - 2 * hexp.Ly) < 1e-4
    pos, n = hex_walkers(hexp, [40], seed=4)
    C = W.cartesian(hexp, pos[0, :n[0]])
    A2 = np.array([hexp.shear * hexp.Ly, hexp.Ly, 0.0])
    both = np.concatenate([C, C + A2])
    both[:, 0] = np.mod(both[:, 0], rect.Lx)
    both[:, 1] = np.mod(both[:, 1], rect.Ly)
    rpos = np.zeros((1, rect.nmax, 3))
    rpos[0, :2 * n[0]] = both
    e_hex = O.Oracle(hexp, pos=pos, n=n).energy[0]
    # the rectangular cell's own slab: same lattice, same origin
    e_rect = O.Oracle(rect, pos=rpos, n=np.array([2 * n[0]], np.int32)).energy[0]
    # the two descriptions round their coordinates to binary32 separately:
    # equal up to that rounding (a geometry mistake costs far more)
    assert abs(e_rect - 2.0 * e_hex) < 1e-7 * max(1.0, abs(e_rect)), (e_rect, e_hex)


def test_forces_are_minus_the_cartesian_gradient():
    p = W.lj_a18_hex_slab(L=1, M=1, nmax=32, seed=5)
    pos, n = hex_walkers(p, [14], seed=6)
    o = O.Oracle(p, pos=pos, n=n)
    f = o.forces(0)
    h = 1e-6
    s = p.shear
    for i in range(int(n[0])):
        g = []
        for c in range(2):                      # d E / d u and d E / d v at fixed other cell coordinates
            save = o.pos[0, i, c]
            o.pos[0, i, c] = save + h
            ep = o.total_energy(0)
            o.pos[0, i, c] = save - h
            em = o.total_energy(0)
            o.pos[0, i, c] = save
            g.append((ep - em) / (2 * h))
        # x = u + s v, y = v: dE/du = dE/dx, dE/dv = s dE/dx + dE/dy
        fx, fy = -g[0], -(g[1] - s * g[0])
        for got, want in ((f[i, 0], fx), (f[i, 1], fy)):
            assert abs(got - want) <= 1e-5 * max(1.0, abs(want)), (i, got, want)


def test_one_particle_canonical_energy_by_quadrature():
    """N = 1 fixed (displacements only, 2.5 A zone): <E> from the oracle's
    Metropolis chain in the cell frame against the midpoint quadrature of
    exp(-beta e_s) over the cell (uniform measure du dv dz, the area Lx Ly)."""
    base = W.lj_a18_hex_slab(L=1, M=1, nmax=2, zone=2.5, seed=7)
    kT = W.K_B_EV * 2500.0                      # hot enough to leave the hollows often
    p = base.replace(kT=np.array([kT]), p_disp=1.0, max_disp=0.5, moves_per_sweep=20)
    nu, nv, nz = 72, 64, 40
    u = (np.arange(nu) + 0.5) * p.Lx / nu
    v = (np.arange(nv) + 0.5) * p.Ly / nv
    z = p.z_lo + (np.arange(nz) + 0.5) * (p.z_hi - p.z_lo) / nz
    U, V, Z = np.meshgrid(u, v, z, indexing="ij")
    pts = np.stack([U.ravel(), V.ravel(), Z.ravel()], 1)
    A1 = np.array([p.Lx, 0.0, 0.0])
    A2 = np.array([p.shear * p.Ly, p.Ly, 0.0])
    shifts = np.array([i * A1 + j * A2 for i in range(-2, 3) for j in range(-2, 3)])
    Cp = W.cartesian(p, pts)
    Sx = W.cartesian(p, p.surf_xyz)
    es = np.zeros(len(pts))
    for a in Sx:
        for sh in shifts:
            d = Cp - (a + sh)
            es += lj(np.sum(d * d, axis=1), p.eps[0, 1], p.sigma[0, 1], p.rc)
    wq = np.exp(-(es - es.min()) / kT)
    e_quad = float((es * wq).sum() / wq.sum())
    pos = np.zeros((1, p.nmax, 3))
    pos[0, 0] = W.f32([p.Lx / 2, p.Ly / 2, p.z_lo + 1.0])
    o = O.Oracle(p, pos=pos, n=np.array([1], np.int32))
    o.sweeps(200, hist=False)
    batches = []
    for b in range(20):
        m0, om0 = o.moments.copy(), o.omega.copy()
        o.sweeps(600)
        batches.append((o.moments[0, 2] - m0[0, 2]) / (o.omega[0] - om0[0]))
    batches = np.array(batches)
    zsc = (batches.mean() - e_quad) / (batches.std(ddof=1) / math.sqrt(len(batches)))
    assert abs(zsc) < 4.5, (batches.mean(), e_quad, zsc)
