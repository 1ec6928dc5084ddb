"""Thin Python binding of the REGC C ABI (argument marshalling only).

Every step of the sampler and of the reweighting runs in the CUDA library;
this module converts numpy arrays and problem statements to the C structs of
include/regc.h and back.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import check

MOVE_DTYPE = np.dtype([
    ("type", np.int32), ("index", np.int32), ("accepted", np.int32), ("status", np.int32),
    ("dE", np.float64), ("log_alpha", np.float64), ("ln_u", np.float64),
    ("sum_abs", np.float64), ("band", np.float64), ("n_pairs", np.int32), ("stage1", np.int32),
    ("dE_sur", np.float64), ("ln_u1", np.float64),
])
assert MOVE_DTYPE.itemsize == C.sizeof(_lib.MoveRecord)
SURROGATE_PARAMS = _lib.SURROGATE_PARAMS


def _p(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(int(stream.cuda_stream))   # torch.cuda.Stream


class Regc:
    """One REGC run: the walkers of an L x M (kT, mu) grid on one GPU.

    ``problem`` is any object with the fields of a problem statement (potential
    tables eps/sigma/rc/n_types, box Lx/Ly/Lz/periodic_z, region z_lo/z_hi,
    surface surf_xyz/surf_type, grid kT/mu/lambda0, nmax, moves_per_sweep,
    max_disp, p_disp, seed, E-histogram e_lo/e_bin/n_e_bins).  ``stream`` is a
    torch.cuda.Stream, a raw cudaStream_t integer, or None (default stream)."""

    def __init__(self, problem, stream=None):
        L = _lib.lib()
        self.p = problem
        pot = _lib.Potential()
        pot.n_types = int(problem.n_types)
        for i in range(4):
            for j in range(4):
                pot.eps[i][j] = float(problem.eps[i][j])
                pot.sigma[i][j] = float(problem.sigma[i][j])
        pot.rc = float(problem.rc)
        self._sxyz = np.ascontiguousarray(np.asarray(problem.surf_xyz, np.float32).reshape(-1, 3))
        self._stype = np.ascontiguousarray(np.asarray(problem.surf_type, np.int32))
        surf = _lib.Surface(len(self._stype), _p(self._sxyz, C.c_float), _p(self._stype, C.c_int32),
                            float(problem.Lx), float(problem.Ly), float(problem.Lz),
                            int(problem.periodic_z), float(problem.z_lo), float(problem.z_hi),
                            float(getattr(problem, "shear", 0.0)))
        self._kT = np.ascontiguousarray(problem.kT, np.float64)
        self._mu = np.ascontiguousarray(problem.mu, np.float64)
        grid = _lib.GridSpec(len(self._kT), len(self._mu), _p(self._kT, C.c_double),
                             _p(self._mu, C.c_double), float(problem.lambda0), int(problem.nmax),
                             int(problem.moves_per_sweep), float(problem.max_disp),
                             float(problem.p_disp), float(problem.e_lo), float(problem.e_bin),
                             int(problem.n_e_bins))
        h = C.c_void_p()
        self.two = int(getattr(problem, "gc2_type", 0)) > 0
        if self.two:
            self._mu2 = np.ascontiguousarray(problem.mu2, np.float64)
            sp2 = _lib.Species2(int(problem.gc2_type), len(self._mu2), _p(self._mu2, C.c_double),
                                float(problem.lambda0_2))
            check(L.regc_init_grid2(C.byref(pot), C.byref(surf), C.byref(grid), C.byref(sp2),
                                    C.c_uint64(int(problem.seed)), _stream_handle(stream), C.byref(h)),
                  "regc_init_grid2")
        else:
            check(L.regc_init_grid(C.byref(pot), C.byref(surf), C.byref(grid), C.c_uint64(int(problem.seed)),
                                   _stream_handle(stream), C.byref(h)), "regc_init_grid")
        self._h = h
        self.K = len(self._mu2) if self.two else 1
        self.S = len(self._kT) * len(self._mu) * self.K
        self.n_cluster = int(getattr(problem, "n_cluster", 0))
        if self.n_cluster > 0:
            check(L.regc_set_cluster(h, self.n_cluster, int(problem.cluster_type)), "regc_set_cluster")
        self.nmax = int(problem.nmax)
        self.mps = int(problem.moves_per_sweep)
        self.n_e_bins = int(problem.n_e_bins)
        self.hE_bins = 0
        self.shard = (0, self.S)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().regc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the sampler
    def sweep(self, n_sweeps: int):
        check(_lib.lib().regc_sweep(self._h, int(n_sweeps)), "regc_sweep")

    def sweep_traced(self, n_sweeps: int) -> np.ndarray:
        tr = np.zeros((self.S, n_sweeps, self.mps), MOVE_DTYPE)
        check(_lib.lib().regc_sweep_traced(self._h, int(n_sweeps), tr.ctypes.data), "regc_sweep_traced")
        return tr

    def exchange(self):
        check(_lib.lib().regc_exchange(self._h), "regc_exchange")

    # -- one grid over several processes (regc_set_shard; see shard.py)
    def set_shard(self, w_begin: int, w_end: int):
        """Step only walkers [w_begin, w_end) from now on."""
        check(_lib.lib().regc_set_shard(self._h, int(w_begin), int(w_end)), "regc_set_shard")
        self.shard = (int(w_begin), int(w_end))

    def walker_ne(self, w_begin: int, w_end: int):
        """(N, N_B or None, exact energies as int64 units of 2^-30) of walkers
        [w_begin, w_end)."""
        k = int(w_end) - int(w_begin)
        n = np.zeros(k, np.int32)
        nb = np.zeros(k, np.int32) if self.two else None
        e = np.zeros(k, np.int64)
        check(_lib.lib().regc_get_walker_ne(self._h, int(w_begin), int(w_end), _p(n, C.c_int32),
                                            _p(nb, C.c_int32),
                                            _p(e, C.c_int64)), "regc_get_walker_ne")
        return n, nb, e

    def set_walker_ne(self, w_begin: int, n, nb, efix):
        """Write another process's walkers' N (N_B) and exact energies from w_begin on."""
        n = np.ascontiguousarray(n, np.int32)
        e = np.ascontiguousarray(efix, np.int64)
        nbc = np.ascontiguousarray(nb, np.int32) if nb is not None else None
        check(_lib.lib().regc_set_walker_ne(self._h, int(w_begin), int(w_begin) + len(n), _p(n, C.c_int32),
                                            _p(nbc, C.c_int32),
                                            _p(e, C.c_int64)), "regc_set_walker_ne")

    def cycle(self, n_steps: int, x0: float, n_canonical: int) -> int:
        """n_steps steps of the REGC cycle (regc_cycle); returns the number of
        replica-exchange steps."""
        n_ex = C.c_int(0)
        check(_lib.lib().regc_cycle(self._h, int(n_steps), float(x0), int(n_canonical), C.byref(n_ex)),
              "regc_cycle")
        return n_ex.value

    def cycle_md(self, n_steps: int, x0: float, md_steps: int, dt: float, tau: float) -> int:
        """REGCMD steps (regc_cycle_md); returns the replica-exchange steps."""
        n_ex = C.c_int(0)
        check(_lib.lib().regc_cycle_md(self._h, int(n_steps), float(x0), int(md_steps), float(dt), float(tau),
                                       C.byref(n_ex)), "regc_cycle_md")
        return n_ex.value

    def cycle_traced(self, n_steps: int, x0: float, n_canonical: int):
        """As cycle, with the trace [S, n_steps, n_canonical + 1]; returns
        (trace, replica-exchange steps)."""
        tr = np.zeros((self.S, n_steps, n_canonical + 1), MOVE_DTYPE)
        n_ex = C.c_int(0)
        check(_lib.lib().regc_cycle_traced(self._h, int(n_steps), float(x0), int(n_canonical), tr.ctypes.data,
                                           C.byref(n_ex)), "regc_cycle_traced")
        return tr, n_ex.value

    def md(self, n_steps: int, dt: float, tau: float, kinetic: bool = True):
        """One MD segment of every walker (regc_md); returns the kinetic
        energies [S] after the last step (or None when kinetic is False)."""
        k = np.zeros(self.S, np.float32) if kinetic else None
        check(_lib.lib().regc_md(self._h, int(n_steps), float(dt), float(tau), _p(k, C.c_float)), "regc_md")
        return k

    def run(self, n_sweeps: int, exchange_every: int = 10):
        """Blocks of exchange_every sweeps, each followed by one exchange attempt."""
        done = 0
        while done < n_sweeps:
            k = min(exchange_every, n_sweeps - done) if exchange_every > 0 else n_sweeps - done
            self.sweep(k)
            done += k
            if exchange_every > 0 and k == exchange_every:
                self.exchange()

    # -- state
    def set_walkers(self, pos, n, state_of_walker=None, nb=None):
        """nb: with a second species, species B's count per walker (particles
        [0, nb[w]) are B); None makes every particle B."""
        pos = np.ascontiguousarray(np.asarray(pos, np.float32).reshape(self.S, self.nmax, 3))
        n = np.ascontiguousarray(np.asarray(n, np.int32))
        sow = None if state_of_walker is None else np.ascontiguousarray(np.asarray(state_of_walker, np.int32))
        nb = None if nb is None else np.ascontiguousarray(np.asarray(nb, np.int32))
        check(_lib.lib().regc_set_walkers2(self._h, _p(pos, C.c_float), _p(n, C.c_int32), _p(nb, C.c_int32),
                                           _p(sow, C.c_int32)), "regc_set_walkers2")

    def species_counts(self) -> np.ndarray:
        """Species B's count N_B per walker (second species only)."""
        nb = np.zeros(self.S, np.int32)
        check(_lib.lib().regc_get_walkers2(self._h, None, None, _p(nb, C.c_int32), None, None), "regc_get_walkers2")
        return nb

    def get_walkers(self, out=None):
        """(pos [S][nmax][3] float32, n [S] int32, energy [S] float64,
        state_of_walker [S] int32); `out` may supply those four arrays (for
        example views of pinned host memory) to be filled in place."""
        if out is None:
            pos = np.zeros((self.S, self.nmax, 3), np.float32)
            n = np.zeros(self.S, np.int32)
            e = np.zeros(self.S)
            sow = np.zeros(self.S, np.int32)
        else:
            pos, n, e, sow = out
            assert pos.dtype == np.float32 and pos.flags.c_contiguous and pos.size == self.S * self.nmax * 3
            assert n.dtype == np.int32 and e.dtype == np.float64 and sow.dtype == np.int32
        check(_lib.lib().regc_get_walkers(self._h, _p(pos, C.c_float), _p(n, C.c_int32), _p(e, C.c_double),
                                          _p(sow, C.c_int32)), "regc_get_walkers")
        return pos, n, e, sow

    def checkpoint(self) -> bytes:
        """The handle's full run state (see regc_checkpoint) as bytes."""
        n = C.c_size_t(0)
        check(_lib.lib().regc_checkpoint(self._h, None, 0, C.byref(n)), "regc_checkpoint")
        buf = C.create_string_buffer(n.value)
        check(_lib.lib().regc_checkpoint(self._h, buf, n.value, C.byref(n)), "regc_checkpoint")
        return buf.raw[:n.value]

    def restore(self, data: bytes):
        buf = C.create_string_buffer(bytes(data), len(data))
        check(_lib.lib().regc_restore(self._h, buf, len(data)), "regc_restore")

    def check_energy(self) -> float:
        d = C.c_double(0)
        check(_lib.lib().regc_check_energy(self._h, C.byref(d)), "regc_check_energy")
        return d.value

    # -- structural observables (axial density, lateral RDF; MBAR per phase)
    def structure_init(self, n_z: int, dz: float, layers, n_r: int, dr: float, capacity: int):
        """layers: up to four (z_lo, z_hi) windows for the lateral RDF."""
        layers = list(layers)
        spec = _lib.StructureSpec()
        spec.n_z, spec.dz, spec.n_layers, spec.n_r, spec.dr = int(n_z), float(dz), len(layers), int(n_r), float(dr)
        for l, (lo, hi) in enumerate(layers):
            spec.layer_lo[l], spec.layer_hi[l] = float(lo), float(hi)
        spec.capacity = int(capacity)
        check(_lib.lib().regc_structure_init(self._h, C.byref(spec)), "regc_structure_init")
        self._stc = (int(n_z), len(layers), int(n_r))

    def structure_sample(self):
        check(_lib.lib().regc_structure_sample(self._h), "regc_structure_sample")

    def structure_count(self) -> int:
        c = C.c_int64(0)
        check(_lib.lib().regc_structure_count(self._h, C.byref(c)), "regc_structure_count")
        return c.value

    def structure_reset(self):
        check(_lib.lib().regc_structure_reset(self._h), "regc_structure_reset")

    def structure_get(self, first: int = 0, count=None) -> dict:
        n_z, n_l, n_r = self._stc
        if count is None:
            count = self.structure_count() - first
        out = {"state": np.zeros(count, np.int32), "N": np.zeros(count, np.int32), "E": np.zeros(count),
               "rho": np.zeros((count, n_z), np.uint16), "pairs": np.zeros((count, n_l, n_r), np.uint32),
               "pop": np.zeros((count, n_l), np.int32)}
        check(_lib.lib().regc_structure_get(self._h, int(first), int(count), out["state"].ctypes.data,
                                            out["N"].ctypes.data, out["E"].ctypes.data, out["rho"].ctypes.data,
                                            out["pairs"].ctypes.data if n_l else None,
                                            out["pop"].ctypes.data if n_l else None), "regc_structure_get")
        return out

    def structure_reweight(self, kT_q, mu_q, n_lo: int, n_hi: int, tol: float = 1e-10, max_iter: int = 200000):
        """MBAR averages per phase N_B = n_lo..n_hi (regc_structure_reweight):
        dict p [Q, P], rho [Q, P, n_z], gxy [Q, P, n_layers, n_r], f [S], iters."""
        n_z, n_l, n_r = self._stc
        kq = np.ascontiguousarray(kT_q, np.float64)
        mq = np.ascontiguousarray(mu_q, np.float64)
        Q, P = len(kq), n_hi - n_lo + 1
        out = {"p": np.zeros((Q, P)), "rho": np.zeros((Q, P, n_z)), "gxy": np.zeros((Q, P, n_l, n_r)),
               "f": np.zeros(self.S)}
        it = C.c_int(0)
        check(_lib.lib().regc_structure_reweight(self._h, Q, _p(kq, C.c_double), _p(mq, C.c_double), int(n_lo),
                                                 int(n_hi), float(tol), int(max_iter), _p(out["p"], C.c_double),
                                                 _p(out["rho"], C.c_double), _p(out["gxy"], C.c_double),
                                                 _p(out["f"], C.c_double), C.byref(it)), "regc_structure_reweight")
        out["iters"] = it.value
        return out

    def aiat(self, mu_q):
        """aiAT@REGC (regc_aiat): (e_min [nmax+1], dG [Q, nmax+1], phase [Q])."""
        mq = np.ascontiguousarray(np.atleast_1d(mu_q), np.float64)
        e_min = np.zeros(self.nmax + 1)
        dG = np.zeros((len(mq), self.nmax + 1))
        ph = np.zeros(len(mq), np.int32)
        check(_lib.lib().regc_aiat(self._h, len(mq), _p(mq, C.c_double), _p(e_min, C.c_double), _p(dG, C.c_double),
                                   ph.ctypes.data), "regc_aiat")
        return e_min, dG, ph

    def aiat_config(self, n_b: int) -> np.ndarray:
        """The lowest-energy sampled configuration with N_B = n_b: [n, 3]."""
        xyz = np.zeros((self.nmax, 3), np.float32)
        n = C.c_int32(0)
        check(_lib.lib().regc_aiat_config(self._h, int(n_b), _p(xyz, C.c_float), C.byref(n)), "regc_aiat_config")
        return xyz[:n.value].copy()

    def structure_timing(self) -> dict:
        v = [C.c_double(0) for _ in range(4)]
        check(_lib.lib().regc_structure_timing(self._h, *[C.byref(x) for x in v]), "regc_structure_timing")
        return {"ms_mbar": v[0].value, "ms_weights": v[1].value, "ms_accumulate": v[2].value,
                "bytes_accumulate": v[3].value}

    def warps_per_walker(self) -> int:
        w = C.c_int(0)
        check(_lib.lib().regc_warps_per_walker(self._h, C.byref(w)), "regc_warps_per_walker")
        return w.value

    def counters(self):
        mv = np.zeros((self.S, 3, 2), np.int64)
        ex = np.zeros((self.S, 5 if self.K > 1 else 4, 2), np.int64)
        pr = np.zeros(6, np.int64)
        check(_lib.lib().regc_counters(self._h, _p(mv, C.c_int64), _p(ex, C.c_int64), _p(pr, C.c_int64)),
              "regc_counters")
        return mv, ex, pr

    # -- learned surrogate (delayed acceptance)
    def surrogate_set(self, theta):
        th = np.ascontiguousarray(np.asarray(theta, np.float32).reshape(SURROGATE_PARAMS))
        check(_lib.lib().regc_surrogate_set(self._h, _p(th, C.c_float)), "regc_surrogate_set")

    def surrogate_init(self, seed: int, scale: float = 1.0):
        check(_lib.lib().regc_surrogate_init(self._h, C.c_uint64(int(seed)), float(scale)), "regc_surrogate_init")

    def surrogate_get(self) -> np.ndarray:
        th = np.zeros(SURROGATE_PARAMS, np.float32)
        check(_lib.lib().regc_surrogate_get(self._h, _p(th, C.c_float)), "regc_surrogate_get")
        return th

    def set_mode(self, delayed: bool):
        check(_lib.lib().regc_set_mode(self._h, 1 if delayed else 0), "regc_set_mode")

    def surrogate_eval(self, walker: int, xyz):
        q = np.ascontiguousarray(np.asarray(xyz, np.float32).reshape(-1, 3))
        e = np.zeros(len(q), np.float32)
        f = np.zeros((len(q), 16), np.float32)
        check(_lib.lib().regc_surrogate_eval(self._h, int(walker), len(q), _p(q, C.c_float), _p(e, C.c_float),
                                             _p(f, C.c_float)), "regc_surrogate_eval")
        return e, f

    def surrogate_harvest(self, particles: int, probes: int, e_clip: float, capacity: int = 0) -> int:
        n = C.c_int64(0)
        check(_lib.lib().regc_surrogate_harvest(self._h, int(particles), int(probes), float(e_clip),
                                                int(capacity), C.byref(n)), "regc_surrogate_harvest")
        return n.value

    def surrogate_set_dataset(self, X, y, capacity: int = 0):
        """Replace the training rows by caller rows X [n, 16], y [n]."""
        X = np.ascontiguousarray(np.asarray(X, np.float32).reshape(-1, 16))
        y = np.ascontiguousarray(np.asarray(y, np.float32).reshape(-1))
        check(_lib.lib().regc_surrogate_set_dataset(self._h, len(y), _p(X, C.c_float), _p(y, C.c_float),
                                                    int(capacity)), "regc_surrogate_set_dataset")

    def surrogate_dataset(self):
        n = C.c_int64(0)
        check(_lib.lib().regc_surrogate_dataset(self._h, 0, None, None, C.byref(n)), "regc_surrogate_dataset")
        X = np.zeros((n.value, 16), np.float32)
        y = np.zeros(n.value, np.float32)
        check(_lib.lib().regc_surrogate_dataset(self._h, n.value, _p(X, C.c_float), _p(y, C.c_float),
                                                C.byref(n)), "regc_surrogate_dataset")
        return X, y

    def surrogate_train(self, steps: int, batch: int, lr: float) -> np.ndarray:
        loss = np.zeros(steps, np.float32)
        check(_lib.lib().regc_surrogate_train(self._h, int(steps), int(batch), float(lr), _p(loss, C.c_float)),
              "regc_surrogate_train")
        return loss

    def histograms(self):
        hN = np.zeros((self.S, self.nmax + 1), np.int64)
        rows = (self.nmax + 1) ** 2 if self.two else self.nmax + 1
        hNE = np.zeros((rows, self.n_e_bins), np.int64)
        om = np.zeros(self.S, np.int64)
        mo = np.zeros((self.S, 4))
        eo = np.zeros(self.S, np.int64)
        check(_lib.lib().regc_histograms(self._h, _p(hN, C.c_int64), _p(hNE, C.c_int64), _p(om, C.c_int64),
                                         _p(mo, C.c_double), _p(eo, C.c_int64)), "regc_histograms")
        out = {"hN": hN, "hNE": hNE, "omega": om, "moments": mo, "e_out": eo}
        if self.two:
            hN2 = np.zeros((self.S, self.nmax + 1), np.int64)
            mo2 = np.zeros((self.S, 2))
            check(_lib.lib().regc_histograms2(self._h, _p(hN2, C.c_int64), _p(mo2, C.c_double)), "regc_histograms2")
            out["hN2"], out["moments2"] = hN2, mo2
        return out

    def reset_histograms(self):
        check(_lib.lib().regc_reset_histograms(self._h), "regc_reset_histograms")

    def set_state_windows(self, n_bins: int, e_bin: float, e_lo=None):
        """Per-state energy windows (regc_set_state_windows); e_lo None centres
        each state's window on its mean observed energy."""
        lo = None if e_lo is None else np.ascontiguousarray(e_lo, np.float64)
        if lo is not None and lo.shape != (self.S,):
            raise ValueError("e_lo must have one origin per state")
        check(_lib.lib().regc_set_state_windows(self._h, int(n_bins), float(e_bin),
                                                 None if lo is None else _p(lo, C.c_double)),
              "regc_set_state_windows")
        self.hE_bins = int(n_bins)

    def state_histograms(self):
        """(hE [S, n_bins + 2], e_lo [S], e_bin): bin 0 below each state's
        window, k + 1 for window bin k, n_bins + 1 beyond it."""
        hE = np.zeros((self.S, self.hE_bins + 2), np.int64)
        lo = np.zeros(self.S)
        eb = C.c_double(0.0)
        check(_lib.lib().regc_state_histograms(self._h, _p(hE, C.c_int64), _p(lo, C.c_double), C.byref(eb)),
              "regc_state_histograms")
        return hE, lo, eb.value

    def reweight(self, kT_q, mu_q, tol: float = 1e-10, max_iter: int = 100000):
        kq = np.ascontiguousarray(kT_q, np.float64)
        mq = np.ascontiguousarray(mu_q, np.float64)
        Q = len(kq)
        nm = np.zeros(Q)
        pN = np.zeros((Q, self.nmax + 1))
        f = np.zeros(self.S)
        it = C.c_int32(0)
        check(_lib.lib().regc_reweight(self._h, Q, _p(kq, C.c_double), _p(mq, C.c_double), tol, max_iter,
                                       _p(nm, C.c_double), _p(pN, C.c_double), _p(f, C.c_double),
                                       C.byref(it)), "regc_reweight")
        return nm, pN, f, it.value

    def test_expire_waits(self):
        """Failure-detection test hook (regc_test_expire_waits): the next sweep's
        bounded waits expire and the handle reports REGC_ETIMEOUT."""
        check(_lib.lib().regc_test_expire_waits(self._h), "regc_test_expire_waits")

    def reweight2(self, kT_q, mu_q, mu2_q, tol: float = 1e-10, max_iter: int = 100000):
        """Two species: (NB_mean, NC_mean, pNB, pNC, f_states, iterations) at
        the query states (kT_q, mu_q, mu2_q)."""
        kq = np.ascontiguousarray(kT_q, np.float64)
        mq = np.ascontiguousarray(mu_q, np.float64)
        m2 = np.ascontiguousarray(mu2_q, np.float64)
        Q = len(kq)
        if len(mq) != Q or len(m2) != Q:
            raise ValueError("query arrays differ in length")
        nb, nc = np.zeros(Q), np.zeros(Q)
        pb, pc = np.zeros((Q, self.nmax + 1)), np.zeros((Q, self.nmax + 1))
        f = np.zeros(self.S)
        it = C.c_int32(0)
        d = C.c_double
        check(_lib.lib().regc_reweight2(self._h, Q, _p(kq, d), _p(mq, d), _p(m2, d), tol, max_iter, _p(nb, d),
                                        _p(nc, d), _p(pb, d), _p(pc, d), _p(f, d), C.byref(it)), "regc_reweight2")
        return nb, nc, pb, pc, f, it.value


class Batch:
    """Several Regc handles (systems of uneven size) stepped together: one
    step = sweeps_per_step sweeps + one exchange attempt of every member,
    bit-identical to stepping the members one by one."""

    def __init__(self, members, sweeps_per_step: int = 10, stream=None):
        self.members = list(members)          # the members must outlive the batch
        arr = (C.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        b = C.c_void_p()
        check(_lib.lib().regc_batch_create(arr, len(self.members), int(sweeps_per_step), _stream_handle(stream),
                                           C.byref(b)), "regc_batch_create")
        self._b = b
        self.sweeps_per_step = int(sweeps_per_step)

    def run(self, n_steps: int = 1):
        check(_lib.lib().regc_batch_run(self._b, int(n_steps)), "regc_batch_run")

    def autotune(self, rounds: int = 1):
        check(_lib.lib().regc_batch_autotune(self._b, int(rounds)), "regc_batch_autotune")

    def sync(self):
        check(_lib.lib().regc_batch_sync(self._b), "regc_batch_sync")

    def plan(self):
        n = C.c_int(0)
        check(_lib.lib().regc_batch_plan(self._b, 0, C.byref(n), None, None, None, None, None, None),
              "regc_batch_plan")
        k = n.value
        nm, wk, wpc, wpw, ctas = (np.zeros(k, np.int32) for _ in range(5))
        ms = np.zeros(k)
        check(_lib.lib().regc_batch_plan(self._b, k, C.byref(n), _p(nm, C.c_int32), _p(wk, C.c_int32),
                                         _p(wpc, C.c_int32), _p(wpw, C.c_int32), _p(ctas, C.c_int32),
                                         _p(ms, C.c_double)),
              "regc_batch_plan")
        return [{"nmax": int(nm[i]), "walkers": int(wk[i]), "walkers_per_cta": int(wpc[i]),
                 "warps_per_walker": int(wpw[i]), "ctas": int(ctas[i]), "ms": float(ms[i])} for i in range(k)]

    def close(self):
        if getattr(self, "_b", None):
            _lib.lib().regc_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def surrogate_gradient(theta, X, y, stream=None, tensor_cores: bool = False):
    """Mean squared error of the surrogate with parameters theta on rows (X, y)
    and its gradient, from the library's training kernels: binary32 on the
    FP32 pipe, or (tensor_cores) BF16 operands with FP32 accumulation as
    training computes it."""
    th = np.ascontiguousarray(np.asarray(theta, np.float32).reshape(SURROGATE_PARAMS))
    X = np.ascontiguousarray(np.asarray(X, np.float32).reshape(-1, 16))
    y = np.ascontiguousarray(np.asarray(y, np.float32).reshape(-1))
    g = np.zeros(SURROGATE_PARAMS, np.float32)
    loss = C.c_float(0)
    name = "regc_surrogate_gradient_bf16" if tensor_cores else "regc_surrogate_gradient"
    check(getattr(_lib.lib(), name)(len(y), _p(th, C.c_float), _p(X, C.c_float), _p(y, C.c_float),
                                    C.byref(loss), _p(g, C.c_float), _stream_handle(stream)), name)
    return float(loss.value), g


def mbar_solve(kT, mu, lambda0, omega, N_b, E_b, H_b, tol=1e-10, max_iter=100000, stream=None):
    """Device MBAR solve over pooled bins; returns (f [S], D [B], iterations)."""
    kT = np.ascontiguousarray(kT, np.float64)
    mu = np.ascontiguousarray(mu, np.float64)
    om = np.ascontiguousarray(omega, np.float64)
    N_b = np.ascontiguousarray(N_b, np.int32)
    E_b = np.ascontiguousarray(E_b, np.float64)
    H_b = np.ascontiguousarray(H_b, np.float64)
    S, B = len(kT), len(N_b)
    f = np.zeros(S)
    D = np.zeros(B)
    it = C.c_int32(0)
    check(_lib.lib().regc_mbar_solve(S, _p(kT, C.c_double), _p(mu, C.c_double), float(lambda0),
                                     _p(om, C.c_double), B, _p(N_b, C.c_int32), _p(E_b, C.c_double),
                                     _p(H_b, C.c_double), tol, max_iter, _p(f, C.c_double),
                                     _p(D, C.c_double), C.byref(it), _stream_handle(stream)),
          "regc_mbar_solve")
    return f, D, it.value


def mbar_last_info() -> dict:
    """What this thread's last MBAR solve did (regc_mbar_last_info): path 1
    on the sparse kernel matrix, 0 on log-sum-exps only; iterations, matrix
    builds, maps on log-sum-exps, kept entries, S, B, device milliseconds of
    the builds and of the maps on the matrix, the number of those maps, and
    the coarse warm-start solve's iterations, bins, builds and maps."""
    i = _lib.MbarInfo()
    check(_lib.lib().regc_mbar_last_info(C.byref(i)), "regc_mbar_last_info")
    return {k: getattr(i, k) for k, _ in _lib.MbarInfo._fields_}


def mbar_query(kT_q, mu_q, lambda0, N_b, E_b, H_b, D, nmax, stream=None):
    """Device MBAR reweighting to query states; returns (<N> [Q], p_N [Q, nmax+1], f_q [Q])."""
    kq = np.ascontiguousarray(kT_q, np.float64)
    mq = np.ascontiguousarray(mu_q, np.float64)
    N_b = np.ascontiguousarray(N_b, np.int32)
    E_b = np.ascontiguousarray(E_b, np.float64)
    H_b = np.ascontiguousarray(H_b, np.float64)
    D = np.ascontiguousarray(D, np.float64)
    Q = len(kq)
    nm = np.zeros(Q)
    pN = np.zeros((Q, nmax + 1))
    fq = np.zeros(Q)
    check(_lib.lib().regc_mbar_query(Q, _p(kq, C.c_double), _p(mq, C.c_double), float(lambda0), len(N_b),
                                     _p(N_b, C.c_int32), _p(E_b, C.c_double), _p(H_b, C.c_double),
                                     _p(D, C.c_double), int(nmax), _p(nm, C.c_double), _p(pN, C.c_double),
                                     _p(fq, C.c_double), _stream_handle(stream)), "regc_mbar_query")
    return nm, pN, fq


def mbar_solve_static(kT, mu, lambda0, omega, N_b, E_b, H_b, tol=1e-10, max_iter=100000, stream=None):
    """As mbar_solve, through regc_mbar_solve_static: no device memory is
    allocated; the library's fixed scratch area is used instead (at most
    4096 states and 262144 bins; calls that overlap on the GPU race)."""
    kT = np.ascontiguousarray(kT, np.float64)
    mu = np.ascontiguousarray(mu, np.float64)
    om = np.ascontiguousarray(omega, np.float64)
    N_b = np.ascontiguousarray(N_b, np.int32)
    E_b = np.ascontiguousarray(E_b, np.float64)
    H_b = np.ascontiguousarray(H_b, np.float64)
    S, B = len(kT), len(N_b)
    f = np.zeros(S)
    D = np.zeros(B)
    it = C.c_int32(0)
    check(_lib.lib().regc_mbar_solve_static(S, _p(kT, C.c_double), _p(mu, C.c_double), float(lambda0),
                                            _p(om, C.c_double), B, _p(N_b, C.c_int32), _p(E_b, C.c_double),
                                            _p(H_b, C.c_double), tol, max_iter, _p(f, C.c_double),
                                            _p(D, C.c_double), C.byref(it), _stream_handle(stream)),
          "regc_mbar_solve_static")
    return f, D, it.value


def mu_of_pressure(kT, p, lambda0: float) -> np.ndarray:
    """mu = kT (3 ln Lambda + ln(p / kT)) of the ideal-gas reservoir (regc_mu_of_pressure)."""
    kT = np.ascontiguousarray(np.atleast_1d(kT), np.float64)
    p = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(p), kT.shape), np.float64)
    mu = np.zeros_like(kT)
    check(_lib.lib().regc_mu_of_pressure(len(kT), _p(kT, C.c_double), _p(p, C.c_double), float(lambda0),
                                         _p(mu, C.c_double)), "regc_mu_of_pressure")
    return mu


def pressure_of_mu(kT, mu, lambda0: float) -> np.ndarray:
    """p = (kT / Lambda^3) exp(mu / kT) of the ideal-gas reservoir (regc_pressure_of_mu)."""
    kT = np.ascontiguousarray(np.atleast_1d(kT), np.float64)
    mu = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(mu), kT.shape), np.float64)
    p = np.zeros_like(kT)
    check(_lib.lib().regc_pressure_of_mu(len(kT), _p(kT, C.c_double), _p(mu, C.c_double), float(lambda0),
                                         _p(p, C.c_double)), "regc_pressure_of_mu")
    return p
