"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module builds problem statements (surface slab, box, gas region, (T, mu)
grid, move settings) and seeded initial walker configurations.  It holds none
of the sampler's arithmetic: no pair potential, no acceptance rule, no random
stream of the method.  Every geometric value is rounded to binary32 here, once,
so that the FP64 oracle and the FP32 GPU path start from identical numbers.

Workloads (reduced Lennard-Jones units, k_B = eps_gg = sigma_gg = m = 1):

* ``fcc100_small`` -- frozen fcc(100) slab of 4x4x2 atoms (32 atoms, in-layer
  nearest-neighbour distance 1.5625), periodic 6.25 x 6.25 box, gas region
  from the top layer to a hard wall at z = 10, eps_sg = 2, rc = 2.5,
  4 kT (0.6-1.5 geometric) x 4 mu (-6..-2), Nmax 32, 20 moves per sweep.
* ``fcc111_paper_scale`` -- frozen fcc(111) slab of 12x12x4 atoms (576 atoms,
  ABC stacking), 18.75 x 16.238 box, gas region 12 high above the top layer,
  eps_sg in {1, 2, 3}, 32 x 32 (kT, mu) states, Nmax 512.  This stands in for
  the paper's LJ A18 slab in a B gas (Sec. III.A) in reduced units.
* ``lj_a18_slab`` -- the paper's LJ surface system (Sec. III.A) in eV and
  Angstrom: two-layer fcc(111) A slab, B gas in a 48 A zone, 10 T x 16 mu
  replicas, in a rectangular cell holding two of the paper's 3 x 3 cells.
* ``tiny_box`` -- a few surface atoms in a small box, Nmax <= 2, for
  brute-force partition-function checks.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

F32 = np.float32


def f32(x):
    """Round a scalar or array to binary32 and return it as float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@dataclasses.dataclass
class Problem:
    """A REGC problem statement: potential, surface, box, grid, move settings."""

    n_types: int
    eps: np.ndarray          # [4, 4] float64 (binary32 values)
    sigma: np.ndarray        # [4, 4]
    rc: float
    Lx: float
    Ly: float
    Lz: float
    periodic_z: int
    z_lo: float
    z_hi: float
    surf_xyz: np.ndarray     # [n_surf, 3] float64 (binary32 values)
    surf_type: np.ndarray    # [n_surf] int32, values 1..n_types-1
    kT: np.ndarray           # [L] float64
    mu: np.ndarray           # [M] float64
    lambda0: float
    nmax: int
    moves_per_sweep: int
    max_disp: float
    p_disp: float
    seed: int
    e_lo: float
    e_bin: float
    n_e_bins: int
    name: str = "custom"
    # a second mobile species (configuration 5): particles 0..n_cluster-1 of
    # every walker have potential type cluster_type and only displace
    n_cluster: int = 0
    cluster_type: int = 0
    # sheared (oblique) cell: lattice vectors (Lx, 0) and (shear Ly, Ly); every
    # x coordinate is then the cell-frame u = x - shear y
    shear: float = 0.0
    # a second grand-canonical species C of potential type gc2_type (0: none)
    # with chemical potentials mu2 [K] on a third grid axis (state
    # s = (l M + m) K + k) and thermal wavelength lambda0_2 / sqrt(kT); a
    # walker's particles [0, N_B) are species B, [N_B, N) species C
    gc2_type: int = 0
    mu2: np.ndarray = None
    lambda0_2: float = 1.0

    def __post_init__(self):
        # the C ABI carries these as binary32: round them here, once, so that
        # both implementations start from the same numbers
        for k in ("rc", "Lx", "Ly", "Lz", "z_lo", "z_hi", "max_disp", "shear"):
            setattr(self, k, float(f32(getattr(self, k))))
        self.eps = f32(self.eps)
        self.sigma = f32(self.sigma)
        self.surf_xyz = f32(np.asarray(self.surf_xyz, dtype=np.float64).reshape(-1, 3))

    @property
    def L(self) -> int:
        return int(len(self.kT))

    @property
    def M(self) -> int:
        return int(len(self.mu))

    @property
    def K(self) -> int:
        return int(len(self.mu2)) if self.gc2_type else 1

    @property
    def S(self) -> int:
        return self.L * self.M * self.K

    def state_params(self):
        """Per state s: (kT, mu, mu2) with s = (l M + m) K + k."""
        s = np.arange(self.S)
        kT = np.asarray(self.kT)[s // (self.M * self.K)]
        mu = np.asarray(self.mu)[(s // self.K) % self.M]
        mu2 = np.asarray(self.mu2)[s % self.K] if self.gc2_type else np.zeros(self.S)
        return kT, mu, mu2

    @property
    def n_surf(self) -> int:
        return int(len(self.surf_type))

    @property
    def volume(self) -> float:
        return self.Lx * self.Ly * (self.z_hi - self.z_lo)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _pair_tables(eps_gg, sig_gg, eps_sg, sig_sg):
    eps = np.zeros((4, 4))
    sig = np.ones((4, 4))
    eps[0, 0] = eps_gg
    sig[0, 0] = sig_gg
    eps[0, 1] = eps[1, 0] = eps_sg
    sig[0, 1] = sig[1, 0] = sig_sg
    return f32(eps), f32(sig)


def fcc100_slab(nx: int, ny: int, layers: int, s: float):
    """fcc(100) slab: square in-layer lattice of spacing s, alternate layers
    shifted by (s/2, s/2), layer spacing s/sqrt(2).  Returns (xyz, Lx, Ly, z_top)."""
    dz = s / math.sqrt(2.0)
    pts = []
    for k in range(layers):
        off = 0.5 * s if (k % 2) else 0.0
        for j in range(ny):
            for i in range(nx):
                pts.append(((i * s + off) % (nx * s), (j * s + off) % (ny * s), k * dz))
    xyz = f32(np.array(pts))
    return xyz, float(f32(nx * s)), float(f32(ny * s)), float(f32((layers - 1) * dz))


def fcc111_slab(nx: int, ny: int, layers: int, s: float):
    """fcc(111) slab in a rectangular supercell of nx columns and ny (even) rows
    of a hexagonal layer with nearest-neighbour distance s; ABC stacking with
    layer spacing s*sqrt(2/3).  Returns (xyz, Lx, Ly, z_top)."""
    if ny % 2:
        raise ValueError("fcc111_slab needs an even number of rows")
    h = s * math.sqrt(3.0) / 2.0
    lx, ly = nx * s, ny * h
    dz = s * math.sqrt(2.0 / 3.0)
    shifts = [(0.0, 0.0), (0.5 * s, h / 3.0), (s, 2.0 * h / 3.0)]
    pts = []
    for k in range(layers):
        sx, sy = shifts[k % 3]
        for j in range(ny):
            for i in range(nx):
                x = i * s + (0.5 * s if (j % 2) else 0.0) + sx
                y = j * h + sy
                pts.append((x % lx, y % ly, k * dz))
    xyz = f32(np.array(pts))
    xyz[:, 0] = np.where(xyz[:, 0] >= f32(lx), 0.0, xyz[:, 0])
    xyz[:, 1] = np.where(xyz[:, 1] >= f32(ly), 0.0, xyz[:, 1])
    return xyz, float(f32(lx)), float(f32(ly)), float(f32((layers - 1) * dz))


def kT_grid(L: int, lo: float = 0.6, hi: float = 1.5) -> np.ndarray:
    if L == 1:
        return np.array([lo])
    return lo * (hi / lo) ** (np.arange(L) / (L - 1))


def mu_grid(M: int, lo: float = -6.0, hi: float = -2.0) -> np.ndarray:
    if M == 1:
        return np.array([lo])
    return lo + (hi - lo) * np.arange(M) / (M - 1)


def centred_e_lo(lo: float, e_bin: float) -> float:
    """Lower edge of an energy-histogram window at or below lo, placed so that
    E = 0 -- the energy of every empty walker -- is the centre of a bin rather
    than an edge: binned MBAR takes a bin's energy at its centre, and with 0 on
    an edge every empty walker would carry e_bin / 2."""
    return -(math.ceil(-lo / e_bin - 1e-9) + 0.5) * e_bin


def fcc100_small(L: int = 4, M: int = 4, nmax: int = 32, eps_sg: float = 2.0,
                 seed: int = 0) -> Problem:
    """The 16-replica fcc(100) workload (4x4x2 slab, 6.25 x 6.25 x 10 box)."""
    xyz, lx, ly, ztop = fcc100_slab(4, 4, 2, 1.5625)
    eps, sig = _pair_tables(1.0, 1.0, eps_sg, 1.0)
    return Problem(
        n_types=2, eps=eps, sigma=sig, rc=2.5, Lx=lx, Ly=ly, Lz=10.0, periodic_z=0,
        z_lo=ztop, z_hi=10.0, surf_xyz=xyz, surf_type=np.ones(len(xyz), np.int32),
        kT=kT_grid(L), mu=mu_grid(M), lambda0=1.0, nmax=nmax, moves_per_sweep=20,
        max_disp=0.2, p_disp=1.0 / 3.0, seed=seed,
        e_lo=centred_e_lo(-float(nmax) * 12.0, 0.05), e_bin=0.05,
        n_e_bins=int(round(float(nmax) * 13.0 / 0.05)), name="fcc100_small")


def fcc111_paper_scale(L: int = 32, M: int = 32, nmax: int = 512, eps_sg: float = 2.0,
                       seed: int = 0) -> Problem:
    """The 1024-replica fcc(111) workload (12x12x4 slab, gas 12 high, Nmax 512)."""
    xyz, lx, ly, ztop = fcc111_slab(12, 12, 4, 1.5625)
    eps, sig = _pair_tables(1.0, 1.0, eps_sg, 1.0)
    zhi = float(f32(ztop + 12.0))
    return Problem(
        n_types=2, eps=eps, sigma=sig, rc=2.5, Lx=lx, Ly=ly, Lz=zhi, periodic_z=0,
        z_lo=ztop, z_hi=zhi, surf_xyz=xyz, surf_type=np.ones(len(xyz), np.int32),
        kT=kT_grid(L), mu=mu_grid(M), lambda0=1.0, nmax=nmax, moves_per_sweep=20,
        max_disp=0.2, p_disp=1.0 / 3.0, seed=seed,
        e_lo=centred_e_lo(-float(nmax) * 14.0, 0.5), e_bin=0.5,
        n_e_bins=int(round(float(nmax) * 15.0 / 0.5)), name="fcc111_paper_scale")


# Physical constants (CODATA 2018) for the workload in physical units.
K_B_EV = 8.617333262e-5          # Boltzmann constant, eV / K
PLANCK_J_S = 6.62607015e-34
AMU_KG = 1.66053906660e-27
EV_J = 1.602176634e-19


ATM_EV_PER_A3 = 101325.0 / EV_J * 1e-30    # 1 atm in eV / A^3


def mass_from_state_point(T_K: float, p_atm: float, mu_eV: float) -> float:
    """The gas mass (u) for which the ideal-gas reservoir of Sec. III.A maps
    (T, p) onto mu: mu = kT (3 ln Lambda + ln(p / kT)) fixes Lambda, and
    Lambda = h / sqrt(2 pi m kT) fixes m."""
    kT = K_B_EV * T_K
    ln_lam = (mu_eV / kT - math.log(p_atm * ATM_EV_PER_A3 / kT)) / 3.0
    lam_m = math.exp(ln_lam) * 1e-10
    return PLANCK_J_S ** 2 / (2.0 * math.pi * kT * EV_J * lam_m ** 2) / AMU_KG


# The paper does not give the mass of B, but states that (200 K, 2.03e-17 atm)
# is exactly its corner state (200 K, -0.9 eV): that fixes m_B = 16.48 u.
PAPER_B_MASS_AMU = mass_from_state_point(200.0, 2.03e-17, -0.9)


def thermal_lambda0(mass_amu: float) -> float:
    """lambda0 in Angstrom eV^(1/2) such that Lambda(kT) = h / sqrt(2 pi m kT)
    = lambda0 / sqrt(kT) with kT in eV (Sec. II.A.1, the thermal wavelength)."""
    return PLANCK_J_S / math.sqrt(2.0 * math.pi * mass_amu * AMU_KG * EV_J) * 1e10


def lj_a18_slab(L: int = 10, M: int = 16, nmax: int = 256, mass_amu: float = PAPER_B_MASS_AMU,
                rc_over_sigma_ab: float = 2.5, zone: float = 48.0, seed: int = 0) -> Problem:
    """The paper's Lennard-Jones surface system (Sec. III.A, Appendix) in
    physical units: energies in eV, lengths in Angstrom, kT = k_B T in eV.

    A frozen two-layer fcc(111) slab of species A (type 1) with hexagonal
    lattice vectors of 11.489 A for its 3 x 3 cell (nearest-neighbour distance
    11.489 / 3), under a gas of species B (type 0): eps_AB = 0.66 eV,
    eps_BB = 0.01 eV, sigma_AB = 1.91 A, sigma_BB = 1.2 A.  The periodic cell
    here is rectangular, 3 x 6 rows (11.489 x 19.899 A), and holds two of the
    paper's hexagonal 3 x 3 cells: 36 A atoms, so that N_B here corresponds to
    2 N_B of the paper's A18.  B lives in a zone of height `zone` above the
    topmost A layer (hard walls at both ends).  The (T, mu) grid: L
    temperatures from 200 K in steps of 50 K, M chemical potentials from
    -2.4 eV in steps of 0.1 eV (10 x 16 = 160 replicas in the paper).
    The paper gives no cutoff: rc = 2.5 sigma_AB is this workload's choice.
    The mass of B follows from the paper's own (T, p) <-> (T, mu) state point
    (PAPER_B_MASS_AMU, 16.48 u)."""
    s = 11.489 / 3.0
    xyz, lx, ly, ztop = fcc111_slab(3, 6, 2, s)
    eps = np.zeros((4, 4))
    sig = np.ones((4, 4))
    eps[0, 0], sig[0, 0] = 0.01, 1.2
    eps[0, 1] = eps[1, 0] = 0.66
    sig[0, 1] = sig[1, 0] = 1.91
    sig[1, 1] = 2.5
    zhi = float(f32(ztop + zone))
    return Problem(
        n_types=2, eps=f32(eps), sigma=f32(sig), rc=rc_over_sigma_ab * 1.91, Lx=lx, Ly=ly, Lz=zhi,
        periodic_z=0, z_lo=ztop, z_hi=zhi, surf_xyz=xyz, surf_type=np.ones(len(xyz), np.int32),
        kT=K_B_EV * (200.0 + 50.0 * np.arange(L)), mu=-2.4 + 0.1 * np.arange(M),
        lambda0=thermal_lambda0(mass_amu), nmax=nmax, moves_per_sweep=11, max_disp=0.2,
        p_disp=1.0 / 3.0, seed=seed, e_lo=centred_e_lo(-1.8 * nmax, 0.01), e_bin=0.01,
        n_e_bins=int(round(2.0 * nmax / 0.01)), name="lj_a18_slab")


def lj_a18_hex_slab(L: int = 10, M: int = 16, nmax: int = 160, mass_amu: float = PAPER_B_MASS_AMU,
                    rc_over_sigma_ab: float = 2.5, zone: float = 48.0, seed: int = 0) -> Problem:
    """The paper's LJ surface system (Sec. III.A, Appendix) in its own cell:
    the 3 x 3 hexagonal supercell of the fcc(111) layer (lattice vectors of
    11.489 A at 60 degrees), two layers, 18 A atoms, as a sheared cell with
    shear 1/sqrt(3) (x coordinates in the cell frame u = x - y / sqrt(3)).
    Potential, zone, grid, mass and cutoff as in lj_a18_slab."""
    a = 11.489 / 3.0
    h = a * math.sqrt(3.0) / 2.0
    dz = a * math.sqrt(2.0 / 3.0)
    pts = []
    for k, (su, sv) in enumerate(((0.0, 0.0), (a / 3.0, a / (2.0 * math.sqrt(3.0))))):
        for j in range(3):
            for i in range(3):
                pts.append((i * a + su, j * h + sv, k * dz))
    xyz = f32(np.array(pts))
    ref = lj_a18_slab(L=L, M=M, nmax=nmax, mass_amu=mass_amu, rc_over_sigma_ab=rc_over_sigma_ab, zone=zone,
                      seed=seed)
    ztop = float(f32(dz))
    zhi = float(f32(ztop + zone))
    return ref.replace(Lx=3.0 * a, Ly=3.0 * h, Lz=zhi, z_lo=ztop, z_hi=zhi, surf_xyz=xyz,
                       surf_type=np.ones(len(xyz), np.int32), shear=1.0 / math.sqrt(3.0),
                       e_lo=centred_e_lo(-1.8 * nmax, 0.01), e_bin=0.01, n_e_bins=int(round(2.0 * nmax / 0.01)),
                       name="lj_a18_hex")


def hex_hollow_sites(problem: Problem):
    """The 18 hollow sites (both kinds) of the top layer of lj_a18_hex_slab, in
    the cell frame: above the bottom layer's atoms and above the third
    stacking position."""
    a = problem.Lx / 3.0
    h = problem.Ly / 3.0
    pts = []
    for su, sv in ((0.0, 0.0), (2.0 * a / 3.0, a / math.sqrt(3.0))):
        for j in range(3):
            for i in range(3):
                pts.append(((i * a + su) % problem.Lx, (j * h + sv) % problem.Ly))
    xy = f32(np.array(pts))
    xy[:, 0] = np.where(xy[:, 0] >= problem.Lx, 0.0, xy[:, 0])
    xy[:, 1] = np.where(xy[:, 1] >= problem.Ly, 0.0, xy[:, 1])
    return xy


def cartesian(problem: Problem, pos):
    """Cell-frame positions [..., 3] -> Cartesian (x = u + shear y)."""
    out = np.array(pos, np.float64, copy=True)
    out[..., 0] = out[..., 0] + float(getattr(problem, "shear", 0.0)) * out[..., 1]
    return out


def lj_a18_initial(problem: Problem, n_b, seed: int, min_dist: float = 1.9):
    """Seeded walkers of ``lj_a18_slab``: walker w gets n_b[w] B particles,
    the first up to 36 on a random subset of the hollow sites of the top A
    layer (both kinds, 36 in the cell) just above the zone's floor with a small
    random offset, the rest at uniform points of the zone at least min_dist
    from every particle and surface atom.  Binary32 coordinates.
    Returns (pos [S, nmax, 3], n [S])."""
    rng = np.random.default_rng(seed)
    S, nmax = problem.S, problem.nmax
    n_b = np.broadcast_to(np.asarray(n_b, dtype=np.int64), (S,))
    shear = float(getattr(problem, "shear", 0.0))
    if shear != 0.0:
        sites = hex_hollow_sites(problem)
    else:
        s = 11.489 / 3.0
        h = s * math.sqrt(3.0) / 2.0
        sites = []
        for sx, sy in ((0.0, 0.0), (s, 2.0 * h / 3.0)):      # the two hollow sites of a B-stacked top layer
            for j in range(6):
                for i in range(3):
                    sites.append((((i * s + (0.5 * s if j % 2 else 0.0) + sx) % problem.Lx),
                                  (j * h + sy) % problem.Ly))
        sites = np.array(sites)
    box = np.array([problem.Lx, problem.Ly, problem.Lz])
    per = np.array([True, True, False])
    pos = np.zeros((S, nmax, 3))
    n = np.zeros(S, np.int32)
    for w in range(S):
        k = int(min(n_b[w], len(sites)))
        pick = rng.permutation(len(sites))[:k]
        pts = []
        for a in pick:
            x = (sites[a, 0] + rng.uniform(-0.1, 0.1)) % problem.Lx
            y = (sites[a, 1] + rng.uniform(-0.1, 0.1)) % problem.Ly
            q = f32([x, y, problem.z_lo + rng.uniform(0.0, 0.3)])
            q[0] = 0.0 if q[0] >= problem.Lx else q[0]
            q[1] = 0.0 if q[1] >= problem.Ly else q[1]
            pts.append(list(q))
        tries = 0
        while len(pts) < n_b[w] and tries < 200000:
            tries += 1
            q = f32([rng.uniform(0, problem.Lx), rng.uniform(0, problem.Ly),
                     rng.uniform(problem.z_lo + 2.0, problem.z_hi)])
            if q[0] >= problem.Lx or q[1] >= problem.Ly or q[2] > problem.z_hi:
                continue
            others = np.array(pts + [list(a) for a in problem.surf_xyz]).reshape(-1, 3)
            d = q - others
            d = np.where(per, d - box * np.round(d / box), d)
            d[:, 0] += shear * d[:, 1]          # Cartesian x (the reduced image is the nearest within rc)
            if np.min(np.sum(d * d, axis=1)) < min_dist * min_dist:
                continue
            pts.append(list(q))
        if len(pts) < n_b[w]:
            raise ValueError("could not place the requested particles")
        if pts:
            pos[w, :len(pts)] = np.array(pts)
        n[w] = len(pts)
    return pos, n


def tiny_box(nmax: int = 2, rc: float = 1.5, eps_sg: float = 1.0, eps_gg: float = 1.0,
             kT=(1.0,), mu=(-1.0,), seed: int = 0) -> Problem:
    """A 3 x 3 box with two surface atoms under a gas region 1.0 <= z <= 2.6,
    for brute-force partition functions with Nmax <= 2."""
    xyz = f32(np.array([[0.75, 0.75, 0.0], [2.25, 2.25, 0.0]]))
    eps, sig = _pair_tables(eps_gg, 1.0, eps_sg, 1.0)
    return Problem(
        n_types=2, eps=eps, sigma=sig, rc=float(f32(rc)), Lx=3.0, Ly=3.0, Lz=2.6,
        periodic_z=0, z_lo=1.0, z_hi=2.6, surf_xyz=xyz,
        surf_type=np.ones(2, np.int32), kT=np.asarray(kT, float), mu=np.asarray(mu, float),
        lambda0=1.0, nmax=nmax, moves_per_sweep=20, max_disp=0.3, p_disp=1.0 / 3.0,
        seed=seed, e_lo=centred_e_lo(-40.0, 0.05), e_bin=0.05, n_e_bins=1600, name="tiny_box")


def two_gas_small(L: int = 2, M: int = 3, K: int = 3, nmax: int = 32, seed: int = 0) -> Problem:
    """Two reactive gases over configuration 1's fcc(100) slab (the outlook of
    Sec. IV: more than one grand-canonical species): B (type 0: eps_BB 1,
    sigma 1, eps_sB 2) and C (type 2: eps_CC 0.6, sigma_CC 0.9, eps_BC 0.8,
    sigma_BC 0.95, eps_sC 1.2, sigma_sC 0.95, a thermal wavelength 0.7 of B's),
    on an L x M x K grid of kT (0.6 .. 1.5), mu_B (-6 .. -2), mu_C (-6 .. -2)."""
    xyz, lx, ly, ztop = fcc100_slab(4, 4, 2, 1.5625)
    eps = np.zeros((4, 4))
    sig = np.ones((4, 4))
    eps[0, 0], eps[0, 1], eps[1, 0] = 1.0, 2.0, 2.0
    eps[2, 2], sig[2, 2] = 0.6, 0.9
    eps[0, 2] = eps[2, 0] = 0.8
    sig[0, 2] = sig[2, 0] = 0.95
    eps[1, 2] = eps[2, 1] = 1.2
    sig[1, 2] = sig[2, 1] = 0.95
    return Problem(
        n_types=3, eps=f32(eps), sigma=f32(sig), rc=2.5, Lx=lx, Ly=ly, Lz=10.0, periodic_z=0,
        z_lo=ztop, z_hi=10.0, surf_xyz=xyz, surf_type=np.ones(len(xyz), np.int32),
        kT=kT_grid(L), mu=mu_grid(M), lambda0=1.0, nmax=nmax, moves_per_sweep=20,
        max_disp=0.2, p_disp=1.0 / 3.0, seed=seed,
        e_lo=centred_e_lo(-float(nmax) * 12.0, 0.25), e_bin=0.25,
        n_e_bins=int(round(float(nmax) * 13.0 / 0.25)), name="two_gas_small",
        gc2_type=2, mu2=mu_grid(K), lambda0_2=0.7)


def two_gas_paper_scale(L: int = 8, M: int = 16, K: int = 8, nmax: int = 256, seed: int = 0) -> Problem:
    """Two reactive gases over the 1024-replica workload's fcc(111) slab
    (12x12x4, gas 12 high): B and C with two_gas_small's pair parameters,
    eps_sB 2 as in the one-species workload, on an 8 x 16 x 8 grid of kT
    (0.6 .. 1.5), mu_B (-6 .. -2), mu_C (-6 .. -2), N_B + N_C <= 256.  The
    pooled (N_B, N_C, E) histogram (257^2 rows x 3840 bins of 1.0) holds
    2 GB."""
    xyz, lx, ly, ztop = fcc111_slab(12, 12, 4, 1.5625)
    eps = np.zeros((4, 4))
    sig = np.ones((4, 4))
    eps[0, 0], eps[0, 1], eps[1, 0] = 1.0, 2.0, 2.0
    eps[2, 2], sig[2, 2] = 0.6, 0.9
    eps[0, 2] = eps[2, 0] = 0.8
    sig[0, 2] = sig[2, 0] = 0.95
    eps[1, 2] = eps[2, 1] = 1.2
    sig[1, 2] = sig[2, 1] = 0.95
    zhi = float(f32(ztop + 12.0))
    return Problem(
        n_types=3, eps=f32(eps), sigma=f32(sig), rc=2.5, Lx=lx, Ly=ly, Lz=zhi, periodic_z=0,
        z_lo=ztop, z_hi=zhi, surf_xyz=xyz, surf_type=np.ones(len(xyz), np.int32),
        kT=kT_grid(L), mu=mu_grid(M), lambda0=1.0, nmax=nmax, moves_per_sweep=20,
        max_disp=0.2, p_disp=1.0 / 3.0, seed=seed,
        e_lo=centred_e_lo(-float(nmax) * 14.0, 1.0), e_bin=1.0,
        n_e_bins=int(round(float(nmax) * 15.0 / 1.0)), name="two_gas_paper_scale",
        gc2_type=2, mu2=mu_grid(K), lambda0_2=0.7)


def two_gas_initial(problem: Problem, nb, nc, seed: int, min_dist: float = 0.9):
    """Seeded walkers of a two-species problem: walker w holds nb[w]
    particles of B then nc[w] of C at uniform positions of the gas region.
    Returns (pos [S, nmax, 3], n [S], nb [S])."""
    nb = np.broadcast_to(np.asarray(nb, np.int32), (problem.S,)).copy()
    nc = np.broadcast_to(np.asarray(nc, np.int32), (problem.S,)).copy()
    pos, n = initial_walkers(problem, nb + nc, seed=seed, min_dist=min_dist)
    return pos, n, nb


def ideal_gas(problem: Problem) -> Problem:
    """The same problem with every interaction switched off (eps = 0)."""
    return problem.replace(eps=np.zeros((4, 4)), name=problem.name + "_ideal")


def initial_walkers(problem: Problem, n_init, seed: int, min_dist: float = 0.9):
    """Seeded initial configurations: walker w gets n_init[w] particles at
    uniform positions of the gas region, no two closer than min_dist (and no
    particle closer than min_dist to a surface atom), coordinates in binary32.
    Returns (pos [S, nmax, 3] float64, n [S] int32)."""
    rng = np.random.default_rng(seed)
    S, nmax = problem.S, problem.nmax
    n_init = np.broadcast_to(np.asarray(n_init, dtype=np.int64), (S,))
    pos = np.zeros((S, nmax, 3))
    n = np.zeros(S, np.int32)
    box = np.array([problem.Lx, problem.Ly, problem.Lz])
    per = np.array([True, True, bool(problem.periodic_z)])
    for w in range(S):
        pts = []
        tries = 0
        while len(pts) < n_init[w] and tries < 200000:
            tries += 1
            p = f32([rng.uniform(0, problem.Lx), rng.uniform(0, problem.Ly),
                     rng.uniform(problem.z_lo, problem.z_hi)])
            if p[0] >= problem.Lx or p[1] >= problem.Ly or p[2] > problem.z_hi:
                continue
            others = np.array(pts + [list(a) for a in problem.surf_xyz]).reshape(-1, 3)
            if len(others):
                d = p - others
                d = np.where(per, d - box * np.round(d / box), d)
                if np.min(np.sum(d * d, axis=1)) < min_dist * min_dist:
                    continue
            pts.append(list(p))
        if len(pts) < n_init[w]:
            raise ValueError("could not place the requested particles")
        if pts:
            pos[w, :len(pts)] = np.array(pts)
        n[w] = len(pts)
    return pos, n


def lattice_sites(problem: Problem, spacing: float = 1.1, clearance: float = 0.95) -> int:
    """Number of sites lattice_walkers can fill in the problem's region."""
    nx = int(problem.Lx // spacing)
    ny = int(problem.Ly // spacing)
    z0 = problem.z_lo + (0.0 if problem.periodic_z else clearance)
    nz = int((problem.z_hi - 0.05 - z0) // spacing) + 1
    z = z0 + 0.05 + np.arange(nz) * spacing
    return nx * ny * int(np.sum(z <= problem.z_hi - 0.05))


def uneven_batch(n_systems: int = 256, L: int = 4, M: int = 4, seed: int = 0, nmax_exp=(6, 11),
                 side=(6, 16), height=(8.0, 16.0)):
    """The batched uneven workload: n_systems independent systems, each an
    L x M (kT, mu) grid (the grids of fcc100_small) over its own 3-layer
    fcc(100) slab (spacing 1.5625) of nx x ny atoms, nx, ny ~ U{side}, with a
    gas region of height ~ U[height] above the top layer and Nmax = 2^k,
    k ~ U{nmax_exp}.  System i is keyed by seed * 100003 + i.  Returns a list
    of Problems."""
    rng = np.random.default_rng(seed)
    eps, sig = _pair_tables(1.0, 1.0, 2.0, 1.0)
    out = []
    for i in range(n_systems):
        nx, ny = (int(v) for v in rng.integers(side[0], side[1] + 1, size=2))
        h = float(rng.uniform(*height))
        nmax = int(2 ** int(rng.integers(nmax_exp[0], nmax_exp[1] + 1)))
        xyz, lx, ly, ztop = fcc100_slab(nx, ny, 3, 1.5625)
        zhi = float(f32(ztop + h))
        e_bin = max(0.05, nmax / 256.0)
        out.append(Problem(
            n_types=2, eps=eps, sigma=sig, rc=2.5, Lx=lx, Ly=ly, Lz=zhi, periodic_z=0,
            z_lo=ztop, z_hi=zhi, surf_xyz=xyz, surf_type=np.ones(len(xyz), np.int32),
            kT=kT_grid(L), mu=mu_grid(M), lambda0=1.0, nmax=nmax, moves_per_sweep=20,
            max_disp=0.2, p_disp=1.0 / 3.0, seed=seed * 100003 + i,
            e_lo=centred_e_lo(-float(nmax) * 14.0, e_bin), e_bin=e_bin, n_e_bins=int(round(float(nmax) * 15.0 / e_bin)),
            name="uneven_%d" % i))
    return out


def cluster_in_gas(L: int = 64, M: int = 64, nmax_b: int = 64, box: float = 15.0, seed: int = 0) -> Problem:
    """The cluster-in-gas workload: a fully periodic cube of edge `box` with no
    surface, a 4-atom cluster of species A (type 1: eps_AA = 4, sigma_AA = 1.1;
    displacement only) in a gas of species B (type 0: eps_BB = 0.5, sigma_BB =
    1; grand-canonical), eps_AB = 2, sigma_AB = 1, rc = 2.5 for every pair; the
    (kT, mu) grids of fcc100_small with L x M states; Nmax_B = nmax_b."""
    eps = np.zeros((4, 4))
    sig = np.ones((4, 4))
    eps[0, 0] = 0.5
    eps[0, 1] = eps[1, 0] = 2.0
    eps[1, 1] = 4.0
    sig[1, 1] = 1.1
    return Problem(
        n_types=2, eps=eps, sigma=sig, rc=2.5, Lx=box, Ly=box, Lz=box, periodic_z=1,
        z_lo=0.0, z_hi=box, surf_xyz=np.zeros((0, 3)), surf_type=np.zeros(0, np.int32),
        kT=kT_grid(L), mu=mu_grid(M), lambda0=1.0, nmax=nmax_b + 4, moves_per_sweep=20,
        max_disp=0.2, p_disp=1.0 / 3.0, seed=seed,
        e_lo=centred_e_lo(-float(nmax_b) * 16.0 - 40.0, 0.25), e_bin=0.25, n_e_bins=int(round((float(nmax_b) * 17.0 + 40.0) / 0.25)),
        name="cluster_in_gas", n_cluster=4, cluster_type=1)


def cluster_initial(problem: Problem, n_b, seed: int, spacing: float = 1.25):
    """Walkers of a cluster problem: the n_cluster atoms as a regular
    tetrahedron (edge 2^(1/6) sigma_AA) at the box centre (first n_cluster
    slots; a single atom sits at the centre), then n_b[w] B particles on
    jittered lattice sites at least 1.2 from every cluster atom."""
    rng = np.random.default_rng(seed)
    S, nmax, nc = problem.S, problem.nmax, problem.n_cluster
    c = np.array([problem.Lx, problem.Ly, problem.Lz]) / 2.0
    a = 2.0 ** (1.0 / 6.0) * float(problem.sigma[problem.cluster_type, problem.cluster_type])
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * a / (2.0 * math.sqrt(2.0))
    clus = f32(c + (tet[:nc] if nc > 1 else np.zeros((nc, 3))))
    n1 = int(problem.Lx // spacing)
    g = (np.arange(n1) + 0.5) * (problem.Lx / n1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    sites = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if nc:
        d = np.min(np.linalg.norm(sites[:, None, :] - clus[None, :, :], axis=2), axis=1)
        sites = sites[d > 1.2]
    n_b = np.broadcast_to(np.asarray(n_b, np.int64), (S,))
    if n_b.max() + nc > nmax or n_b.max() > len(sites):
        raise ValueError("too many particles")
    pos = np.zeros((S, nmax, 3))
    for w in range(S):
        pos[w, :nc] = clus
        k = int(n_b[w])
        pick = rng.choice(len(sites), size=k, replace=False)
        p = f32((sites[pick] + rng.uniform(-0.05, 0.05, size=(k, 3))) % problem.Lx)
        p = np.where(p >= problem.Lx, 0.0, p)
        pos[w, nc:nc + k] = p
    return pos, (n_b + nc).astype(np.int32)


def uneven_initial(problem: Problem, seed: int):
    """Initial walkers of the batched uneven workload: N ~ U{0..Nmax/2} per
    walker, capped at 90 % of the lattice sites that fit the region (a small
    box cannot hold Nmax/2 particles without overlaps), on the jittered
    lattice of lattice_walkers."""
    rng = np.random.default_rng(seed)
    cap = int(0.9 * lattice_sites(problem))
    n0 = np.minimum(rng.integers(0, problem.nmax // 2 + 1, problem.S), cap)
    return lattice_walkers(problem, n0, seed=seed)


def lattice_walkers(problem: Problem, n_init, seed: int, spacing: float = 1.1,
                    clearance: float = 0.95):
    """Fast seeded initial configurations for large runs: walker w gets
    n_init[w] particles on distinct sites of a simple-cubic lattice of the given
    spacing filling the gas region from z_lo + clearance upward, each site
    jittered by at most 0.05, coordinates in binary32.  No two particles are
    closer than spacing - 0.1.  Returns (pos [S, nmax, 3], n [S] int32)."""
    rng = np.random.default_rng(seed)
    S, nmax = problem.S, problem.nmax
    nx = int(problem.Lx // spacing)
    ny = int(problem.Ly // spacing)
    z0 = problem.z_lo + (0.0 if problem.periodic_z else clearance)
    nz = int((problem.z_hi - 0.05 - z0) // spacing) + 1
    hx, hy = problem.Lx / nx, problem.Ly / ny
    gx, gy, gz = np.meshgrid((np.arange(nx) + 0.5) * hx, (np.arange(ny) + 0.5) * hy,
                             z0 + 0.05 + np.arange(nz) * spacing, indexing="ij")
    sites = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    sites = sites[sites[:, 2] <= problem.z_hi - 0.05]
    n_init = np.broadcast_to(np.asarray(n_init, dtype=np.int64), (S,))
    if n_init.max() > len(sites) or n_init.max() > nmax:
        raise ValueError("too many particles for the lattice or nmax")
    pos = np.zeros((S, nmax, 3))
    for w in range(S):
        k = int(n_init[w])
        pick = rng.choice(len(sites), size=k, replace=False)
        p = sites[pick] + rng.uniform(-0.05, 0.05, size=(k, 3))
        p[:, 0] %= problem.Lx
        p[:, 1] %= problem.Ly
        p = f32(p)
        p[:, 0] = np.where(p[:, 0] >= problem.Lx, 0.0, p[:, 0])
        p[:, 1] = np.where(p[:, 1] >= problem.Ly, 0.0, p[:, 1])
        pos[w, :k] = p
    return pos, n_init.astype(np.int32)
