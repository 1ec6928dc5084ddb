"""Python front end of the FP64 CPU oracle (regc_oracle.c).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
baseline of the benchmark.  The CUDA library never imports or links this.

``build()`` compiles regc_oracle.c with gcc into ``oracle/_build/liboracle.so``
(plain -O2, no fused multiply-add contraction, OpenMP over walkers).  The
``Oracle`` class wraps one problem statement and a set of walkers held in
numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = os.path.join(HERE, "regc_oracle.c")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (a no-op when it is up to date)."""
    os.makedirs(BUILD, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)
            and os.path.getmtime(LIB) >= os.path.getmtime(os.path.join(HERE, "regc_oracle.h"))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _System(C.Structure):
    _fields_ = [
        ("n_types", C.c_int),
        ("eps", (C.c_double * 4) * 4),
        ("sigma", (C.c_double * 4) * 4),
        ("rc", C.c_double),
        ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
        ("periodic_z", C.c_int),
        ("z_lo", C.c_double), ("z_hi", C.c_double),
        ("n_surf", C.c_int),
        ("surf_xyz", C.POINTER(C.c_double)),
        ("surf_type", C.POINTER(C.c_int)),
        ("L", C.c_int), ("M", C.c_int),
        ("kT", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
        ("lambda0", C.c_double),
        ("nmax", C.c_int), ("moves_per_sweep", C.c_int),
        ("max_disp", C.c_double), ("p_disp", C.c_double),
        ("seed", C.c_uint64),
        ("e_lo", C.c_double), ("e_bin", C.c_double),
        ("n_e_bins", C.c_int),
        ("mutation", C.c_int),
        ("da", C.c_int),
        ("sur_theta", C.POINTER(C.c_double)),
        ("n_cluster", C.c_int),
        ("cluster_type", C.c_int),
        ("shear", C.c_double),
        ("gc2_type", C.c_int),
        ("K", C.c_int),
        ("mu2", C.POINTER(C.c_double)),
        ("lambda0_2", C.c_double),
    ]


class _Hist(C.Structure):
    _fields_ = [
        ("hN", C.POINTER(C.c_int64)),
        ("hNE", C.POINTER(C.c_int64)),
        ("omega", C.POINTER(C.c_int64)),
        ("moments", C.POINTER(C.c_double)),
        ("e_out", C.POINTER(C.c_int64)),
        ("hE", C.POINTER(C.c_int64)),
        ("hE_lo", C.POINTER(C.c_double)),
        ("hE_bin", C.c_double),
        ("hE_bins", C.c_int),
        ("hN2", C.POINTER(C.c_int64)),
        ("moments2", C.POINTER(C.c_double)),
    ]


MOVE_DTYPE = np.dtype([
    ("type", np.int32), ("index", np.int32), ("accepted", np.int32), ("status", np.int32),
    ("dE", np.float64), ("log_alpha", np.float64), ("ln_u", np.float64),
    ("sum_abs", np.float64), ("band", np.float64), ("n_pairs", np.int32), ("stage1", np.int32),
    ("dE_sur", np.float64), ("ln_u1", np.float64),
])

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp, ip, i64p = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        sp = C.POINTER(_System)
        _lib.oracle_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        _lib.oracle_phi.argtypes = [sp, C.c_int, C.c_int, C.c_double]
        _lib.oracle_phi.restype = C.c_double
        _lib.oracle_particle_energy.argtypes = [sp, dp, C.c_int, C.c_double, C.c_double,
                                                C.c_double, C.c_int, dp, dp, ip]
        _lib.oracle_particle_energy.restype = C.c_double
        _lib.oracle_total_energy.argtypes = [sp, dp, C.c_int]
        _lib.oracle_total_energy.restype = C.c_double
        _lib.oracle_log_alpha.argtypes = [sp, C.c_int, C.c_int, C.c_int, C.c_double]
        _lib.oracle_log_alpha.restype = C.c_double
        _lib.oracle_exchange_log_alpha.argtypes = [sp, C.c_int, C.c_int, C.c_int, C.c_int,
                                                   C.c_double, C.c_double]
        _lib.oracle_exchange_log_alpha.restype = C.c_double
        _lib.oracle_sweeps.argtypes = [sp, C.c_int, dp, ip, dp, ip, C.c_uint32, C.c_int,
                                       C.POINTER(_Hist), C.c_void_p, i64p, C.c_int]
        _lib.oracle_sweeps.restype = C.c_int
        _lib.oracle_exchange.argtypes = [sp, C.c_uint32, ip, dp, ip, ip, i64p]
        _lib.oracle_exchange.restype = C.c_int
        _lib.oracle_sweeps2.argtypes = [sp, C.c_int, dp, ip, ip, dp, ip, C.c_uint32, C.c_int,
                                        C.POINTER(_Hist), C.c_void_p, i64p, C.c_int]
        _lib.oracle_sweeps2.restype = C.c_int
        _lib.oracle_sweeps_range.argtypes = [sp, C.c_int, dp, ip, ip, dp, ip, C.c_uint32, C.c_int,
                                             C.POINTER(_Hist), C.c_void_p, i64p, C.c_int, C.c_int, C.c_int]
        _lib.oracle_sweeps_range.restype = C.c_int
        _lib.oracle_exchange2.argtypes = [sp, C.c_uint32, ip, ip, dp, ip, ip, i64p]
        _lib.oracle_exchange2.restype = C.c_int
        _lib.oracle_total_energy2.argtypes = [sp, dp, C.c_int, C.c_int]
        _lib.oracle_total_energy2.restype = C.c_double
        _lib.oracle_particle_energy2.argtypes = [sp, dp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                                 C.c_int, C.c_int, dp, dp, ip]
        _lib.oracle_particle_energy2.restype = C.c_double
        _lib.oracle_log_alpha2.argtypes = [sp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double]
        _lib.oracle_log_alpha2.restype = C.c_double
        _lib.oracle_exchange_log_alpha2.argtypes = [sp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                                    C.c_double, C.c_double]
        _lib.oracle_exchange_log_alpha2.restype = C.c_double
        _lib.oracle_surrogate_energy.argtypes = [sp, dp, C.c_int, C.c_double, C.c_double, C.c_double,
                                                 C.c_int, dp]
        _lib.oracle_surrogate_energy.restype = C.c_double
        _lib.oracle_md.argtypes = [sp, C.c_int, dp, ip, dp, ip, C.c_uint32, C.c_int, C.c_double, C.c_double,
                                   dp, C.c_int]
        _lib.oracle_md.restype = C.c_int
        _lib.oracle_cycle.argtypes = [sp, C.c_int, dp, ip, dp, ip, ip, C.c_uint32, C.c_uint32, C.c_int,
                                      C.c_double, C.c_int, C.c_void_p, C.c_void_p, i64p, i64p]
        _lib.oracle_cycle.restype = C.c_int
        _lib.oracle_forces.argtypes = [sp, dp, C.c_int, dp]
        _lib.oracle_forces.restype = None
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr is 4 uint32 words, key is 2."""
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


class Oracle:
    """FP64 REGC sampler over the walkers of one problem statement.

    State (numpy, owned here): pos [S, nmax, 3], n [S], energy [S],
    state_of_walker [S], walker_of_state [S], sweep counter t, exchange
    counter e, histograms and acceptance counters."""

    def __init__(self, problem, pos=None, n=None, mutation: int = 0, n_threads: int = 0,
                 surrogate=None, nb=None):
        self.p = problem
        S, nmax = problem.S, problem.nmax
        self._kT = np.ascontiguousarray(problem.kT, np.float64)
        self._mu = np.ascontiguousarray(problem.mu, np.float64)
        self._sxyz = np.ascontiguousarray(problem.surf_xyz, np.float64).reshape(-1)
        self._stype = np.ascontiguousarray(problem.surf_type, np.int32)
        if len(self._stype) == 0:
            self._sxyz = np.zeros(3)
            self._stype = np.zeros(1, np.int32)
        s = _System()
        s.n_types = problem.n_types
        for i in range(4):
            for j in range(4):
                s.eps[i][j] = float(problem.eps[i, j])
                s.sigma[i][j] = float(problem.sigma[i, j])
        s.rc = problem.rc
        s.Lx, s.Ly, s.Lz = problem.Lx, problem.Ly, problem.Lz
        s.periodic_z = int(problem.periodic_z)
        s.z_lo, s.z_hi = problem.z_lo, problem.z_hi
        s.n_surf = problem.n_surf
        s.surf_xyz = _ptr(self._sxyz, C.c_double)
        s.surf_type = _ptr(self._stype, C.c_int32)
        s.L, s.M = problem.L, problem.M
        s.kT = _ptr(self._kT, C.c_double)
        s.mu = _ptr(self._mu, C.c_double)
        s.lambda0 = problem.lambda0
        s.nmax, s.moves_per_sweep = problem.nmax, problem.moves_per_sweep
        s.max_disp, s.p_disp = problem.max_disp, problem.p_disp
        s.seed = int(problem.seed)
        s.e_lo, s.e_bin, s.n_e_bins = problem.e_lo, problem.e_bin, problem.n_e_bins
        s.mutation = int(mutation)
        s.n_cluster = int(getattr(problem, "n_cluster", 0))
        s.cluster_type = int(getattr(problem, "cluster_type", 0))
        s.shear = float(getattr(problem, "shear", 0.0))
        self.two = int(getattr(problem, "gc2_type", 0)) > 0
        self._mu2 = np.ascontiguousarray(problem.mu2 if self.two else [0.0], np.float64)
        s.gc2_type = int(getattr(problem, "gc2_type", 0))
        s.K = int(problem.K)
        s.mu2 = _ptr(self._mu2, C.c_double)
        s.lambda0_2 = float(getattr(problem, "lambda0_2", 1.0))
        self._theta = None
        if surrogate is not None:
            self._theta = np.ascontiguousarray(surrogate, np.float64)
            s.da = 1
            s.sur_theta = _ptr(self._theta, C.c_double)
        self.sys = s
        self.n_threads = int(n_threads)
        self.pos = np.zeros((S, nmax, 3)) if pos is None else np.array(pos, np.float64).reshape(S, nmax, 3)
        self.n = np.zeros(S, np.int32) if n is None else np.array(n, np.int32)
        # with a second species: N_B per walker (particles [0, N_B) are B)
        self.nb = np.array(self.n if nb is None else nb, np.int32)
        self.energy = np.array([self.total_energy(w) for w in range(S)])
        self.state_of_walker = np.arange(S, dtype=np.int32)
        self.walker_of_state = np.arange(S, dtype=np.int32)
        self.t = 0
        self.e = 0
        self.md_seg = 0
        self.reset_histograms()
        self.counts = np.zeros((S, 3, 2), np.int64)
        self.ex_counts = np.zeros((S, 5 if problem.K > 1 else 4, 2), np.int64)

    def reset_histograms(self):
        p = self.p
        self.hN = np.zeros((p.S, p.nmax + 1), np.int64)
        rows = (p.nmax + 1) ** 2 if getattr(p, "gc2_type", 0) else p.nmax + 1
        self.hNE = np.zeros((rows, p.n_e_bins), np.int64)
        self.hN2 = np.zeros((p.S, p.nmax + 1), np.int64)
        self.moments2 = np.zeros((p.S, 2))
        self.omega = np.zeros(p.S, np.int64)
        self.moments = np.zeros((p.S, 4))
        self.e_out = np.zeros(p.S, np.int64)
        if getattr(self, "hE_lo", None) is not None:
            self.hE = np.zeros((p.S, self.hE.shape[1]), np.int64)

    def set_state_windows(self, n_bins: int, e_bin: float, e_lo):
        """Per-state energy windows: state s has n_bins bins of width e_bin
        from e_lo[s], with an underflow bin first and an overflow bin last."""
        self.hE_lo = np.ascontiguousarray(e_lo, np.float64)
        self.hE_bin = float(e_bin)
        self.hE = np.zeros((self.p.S, int(n_bins) + 2), np.int64)

    def _hist(self):
        h = _Hist(_ptr(self.hN, C.c_int64), _ptr(self.hNE, C.c_int64),
                  _ptr(self.omega, C.c_int64), _ptr(self.moments, C.c_double),
                  _ptr(self.e_out, C.c_int64))
        if self.two:
            h.hN2 = _ptr(self.hN2, C.c_int64)
            h.moments2 = _ptr(self.moments2, C.c_double)
        if getattr(self, "hE_lo", None) is not None:
            h.hE = _ptr(self.hE, C.c_int64)
            h.hE_lo = _ptr(self.hE_lo, C.c_double)
            h.hE_bin = self.hE_bin
            h.hE_bins = self.hE.shape[1] - 2
        return h

    # -- single-function access for the pins
    def phi(self, ti, tj, r2):
        return lib().oracle_phi(C.byref(self.sys), ti, tj, r2)

    def total_energy(self, w):
        pos = np.ascontiguousarray(self.pos[w])
        nb = int(self.nb[w]) if self.two else int(self.n[w])
        return lib().oracle_total_energy2(C.byref(self.sys), _ptr(pos, C.c_double), int(self.n[w]), nb)

    def particle_energy2(self, w, xyz, skip=-1, species_new=0):
        """Interaction energy of a particle at xyz in walker w (two species:
        particles [0, N_B) are B); a new particle has potential type species_new."""
        pos = np.ascontiguousarray(self.pos[w])
        sa, band = C.c_double(0), C.c_double(0)
        npairs = C.c_int32(0)
        e = lib().oracle_particle_energy2(C.byref(self.sys), _ptr(pos, C.c_double), int(self.n[w]),
                                          int(self.nb[w]), float(xyz[0]), float(xyz[1]), float(xyz[2]),
                                          int(skip), int(species_new), C.byref(sa), C.byref(band), C.byref(npairs))
        return e, sa.value, band.value, npairs.value

    def log_alpha2(self, move_type, species, state, n_c, dE):
        return lib().oracle_log_alpha2(C.byref(self.sys), move_type, species, state, n_c, dE)

    def exchange_log_alpha2(self, sa, sb, nba, nca, nbb, ncb, ea, eb):
        return lib().oracle_exchange_log_alpha2(C.byref(self.sys), sa, sb, nba, nca, nbb, ncb, ea, eb)

    def particle_energy(self, w, xyz, skip=-1):
        pos = np.ascontiguousarray(self.pos[w])
        sa, band = C.c_double(0), C.c_double(0)
        npairs = C.c_int32(0)
        e = lib().oracle_particle_energy(C.byref(self.sys), _ptr(pos, C.c_double), int(self.n[w]),
                                         float(xyz[0]), float(xyz[1]), float(xyz[2]), int(skip),
                                         C.byref(sa), C.byref(band), C.byref(npairs))
        return e, sa.value, band.value, npairs.value

    def surrogate_energy(self, w, xyz, skip=-1):
        """Surrogate energy e~ of a particle at xyz in walker w, and its features."""
        if self._theta is None:
            raise ValueError("no surrogate weights")
        pos = np.ascontiguousarray(self.pos[w])
        feat = np.zeros(16)
        e = lib().oracle_surrogate_energy(C.byref(self.sys), _ptr(pos, C.c_double), int(self.n[w]),
                                          float(xyz[0]), float(xyz[1]), float(xyz[2]), int(skip),
                                          _ptr(feat, C.c_double))
        return e, feat

    def log_alpha(self, move_type, state, n, dE):
        return lib().oracle_log_alpha(C.byref(self.sys), move_type, state, n, dE)

    def exchange_log_alpha(self, sa, sb, na, nb, ea, eb):
        return lib().oracle_exchange_log_alpha(C.byref(self.sys), sa, sb, na, nb, ea, eb)

    # -- the sampler
    def sweeps(self, n_sweeps: int, hist: bool = True, trace: bool = False, walkers=None):
        """n_sweeps sweeps of every walker, or of walkers [b, e) given as
        walkers=(b, e) (the others are left as they are)."""
        p = self.p
        S = p.S
        b, e = (0, S) if walkers is None else (int(walkers[0]), int(walkers[1]))
        tr = np.zeros((S, n_sweeps, p.moves_per_sweep), MOVE_DTYPE) if trace else None
        h = None
        if hist:
            h = self._hist()
        rc = lib().oracle_sweeps_range(C.byref(self.sys), S, _ptr(self.pos, C.c_double),
                                  _ptr(self.n, C.c_int32), _ptr(self.nb, C.c_int32) if self.two else None,
                                  _ptr(self.energy, C.c_double),
                                  _ptr(self.state_of_walker, C.c_int32), C.c_uint32(self.t),
                                  n_sweeps, C.byref(h) if h is not None else None,
                                  tr.ctypes.data if tr is not None else None,
                                  _ptr(self.counts, C.c_int64), self.n_threads, b, e)
        if rc != 0:
            raise ValueError("oracle_sweeps rejected its arguments")
        self.t += n_sweeps
        return tr

    def cycle(self, n_steps: int, x0: float, n_canonical: int, hist: bool = True, trace: bool = False):
        """n_steps steps of the REGC cycle (see oracle_cycle): with probability
        x0 one particle-exchange attempt per replica, else one replica-exchange
        attempt; then n_canonical displacement moves per replica.  Returns
        (trace [S, n_steps, n_canonical + 1] or None, replica-exchange steps)."""
        p = self.p
        S = p.S
        tr = np.zeros((S, n_steps, n_canonical + 1), MOVE_DTYPE) if trace else None
        h = None
        if hist:
            h = self._hist()
        n_ex = lib().oracle_cycle(C.byref(self.sys), S, _ptr(self.pos, C.c_double), _ptr(self.n, C.c_int32),
                                  _ptr(self.energy, C.c_double), _ptr(self.state_of_walker, C.c_int32),
                                  _ptr(self.walker_of_state, C.c_int32), C.c_uint32(self.t), C.c_uint32(self.e),
                                  int(n_steps), float(x0), int(n_canonical),
                                  C.cast(C.byref(h), C.c_void_p) if h is not None else None,
                                  tr.ctypes.data if tr is not None else None,
                                  _ptr(self.counts, C.c_int64), _ptr(self.ex_counts, C.c_int64))
        if n_ex < 0:
            raise ValueError("oracle_cycle rejected its arguments")
        self.t += n_steps
        self.e += n_ex
        return tr, n_ex

    def cycle_md(self, n_steps: int, x0: float, md_steps: int, dt: float, tau: float):
        """REGCMD: each step one REGC cycle step without canonical MC moves,
        then one MD segment.  Returns the replica-exchange steps."""
        n_ex = 0
        for _ in range(n_steps):
            n_ex += self.cycle(1, x0, 0)[1]
            self.md(md_steps, dt, tau)
        return n_ex

    def forces(self, w):
        """MD forces [n, 3] on the particles of walker w."""
        n = int(self.n[w])
        pos = np.ascontiguousarray(self.pos[w])
        f = np.zeros((max(n, 1), 3))
        lib().oracle_forces(C.byref(self.sys), _ptr(pos, C.c_double), n, _ptr(f, C.c_double))
        return f[:n]

    def md(self, n_steps: int, dt: float, tau: float):
        """One MD segment of every walker (see oracle_md); returns the kinetic
        energies [S] after the last step."""
        kin = np.zeros(self.p.S)
        pos = np.ascontiguousarray(self.pos)
        rc = lib().oracle_md(C.byref(self.sys), self.p.S, _ptr(pos, C.c_double), _ptr(self.n, C.c_int32),
                             _ptr(self.energy, C.c_double), _ptr(self.state_of_walker, C.c_int32),
                             C.c_uint32(self.md_seg), int(n_steps), float(dt), float(tau),
                             _ptr(kin, C.c_double), self.n_threads)
        if rc < 0:
            raise ValueError("oracle_md rejected its arguments")
        self.pos = pos
        self.md_seg += 1
        return kin

    def exchange(self):
        acc = lib().oracle_exchange2(C.byref(self.sys), C.c_uint32(self.e), _ptr(self.n, C.c_int32),
                                     _ptr(self.nb, C.c_int32) if self.two else None,
                                     _ptr(self.energy, C.c_double),
                                    _ptr(self.state_of_walker, C.c_int32),
                                    _ptr(self.walker_of_state, C.c_int32),
                                    _ptr(self.ex_counts, C.c_int64))
        if acc < 0:
            raise ValueError("oracle_exchange rejected its arguments")
        self.e += 1
        return acc

    def run(self, n_sweeps: int, exchange_every: int = 10, hist: bool = True):
        """Alternate blocks of exchange_every sweeps with an exchange attempt."""
        done = 0
        while done < n_sweeps:
            k = min(exchange_every, n_sweeps - done) if exchange_every > 0 else n_sweeps - done
            self.sweeps(k, hist=hist)
            done += k
            if exchange_every > 0 and k == exchange_every:
                self.exchange()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
