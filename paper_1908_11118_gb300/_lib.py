"""ctypes declarations of the C ABI in include/regc.h.

The shared library is built in-tree (paper_1908_11118_gb300/_build/libregc.so)
by paper_1908_11118_gb300/build.py.  There is no other implementation: if the
library is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libregc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "regc.h")

REGC_OK = 0
STATUS = {0: "REGC_OK", -1: "REGC_EINVAL", -2: "REGC_ENOMEM", -3: "REGC_ECUDA",
          -4: "REGC_ETIMEOUT", -5: "REGC_ECAPACITY", -6: "REGC_ENUMERIC"}


class RegcError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__("%s returned %s" % (where, STATUS.get(status, status)))
        self.status = status


class Potential(C.Structure):
    _fields_ = [("n_types", C.c_int), ("eps", (C.c_float * 4) * 4),
                ("sigma", (C.c_float * 4) * 4), ("rc", C.c_float)]


class Surface(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("xyz", C.POINTER(C.c_float)), ("type", C.POINTER(C.c_int)),
                ("Lx", C.c_float), ("Ly", C.c_float), ("Lz", C.c_float), ("periodic_z", C.c_int),
                ("z_lo", C.c_float), ("z_hi", C.c_float), ("shear", C.c_float)]


class Species2(C.Structure):
    _fields_ = [("type", C.c_int), ("K", C.c_int), ("mu", C.POINTER(C.c_double)), ("lambda0", C.c_double)]


class MbarInfo(C.Structure):
    _fields_ = [("path", C.c_int32), ("iterations", C.c_int32), ("builds", C.c_int32), ("lse_maps", C.c_int32),
                ("nnz", C.c_int64), ("S", C.c_int64), ("B", C.c_int64), ("ms_build", C.c_double),
                ("ms_maps", C.c_double), ("sparse_maps", C.c_int32), ("coarse_iterations", C.c_int32),
                ("coarse_B", C.c_int64), ("coarse_builds", C.c_int32), ("coarse_maps", C.c_int32)]


class GridSpec(C.Structure):
    _fields_ = [("L", C.c_int), ("M", C.c_int), ("kT", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("lambda0", C.c_double), ("nmax", C.c_int),
                ("moves_per_sweep", C.c_int), ("max_disp", C.c_float), ("p_disp", C.c_double),
                ("e_lo", C.c_double), ("e_bin", C.c_double), ("n_e_bins", C.c_int)]


class MoveRecord(C.Structure):
    _fields_ = [("type", C.c_int32), ("index", C.c_int32), ("accepted", C.c_int32),
                ("status", C.c_int32), ("dE", C.c_double), ("log_alpha", C.c_double),
                ("ln_u", C.c_double), ("sum_abs", C.c_double), ("band", C.c_double),
                ("n_pairs", C.c_int32), ("stage1", C.c_int32), ("dE_sur", C.c_double),
                ("ln_u1", C.c_double)]


class StructureSpec(C.Structure):
    _fields_ = [("n_z", C.c_int), ("dz", C.c_float), ("n_layers", C.c_int), ("layer_lo", C.c_float * 4),
                ("layer_hi", C.c_float * 4), ("n_r", C.c_int), ("dr", C.c_float), ("capacity", C.c_int64)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)
_fp = C.POINTER(C.c_float)
_h = C.c_void_p

SIGNATURES = {
    "regc_init_grid": ([C.POINTER(Potential), C.POINTER(Surface), C.POINTER(GridSpec), C.c_uint64,
                        C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "regc_init_grid2": ([C.POINTER(Potential), C.POINTER(Surface), C.POINTER(GridSpec), C.POINTER(Species2),
                         C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "regc_histograms2": ([_h, _lp, _dp], C.c_int),
    "regc_set_walkers2": ([_h, _fp, _ip, _ip, _ip], C.c_int),
    "regc_get_walkers2": ([_h, _fp, _ip, _ip, _dp, _ip], C.c_int),
    "regc_sweep": ([_h, C.c_int], C.c_int),
    "regc_sweep_traced": ([_h, C.c_int, C.c_void_p], C.c_int),
    "regc_exchange": ([_h], C.c_int),
    "regc_set_shard": ([_h, C.c_int, C.c_int], C.c_int),
    "regc_get_walker_ne": ([_h, C.c_int, C.c_int, _ip, _ip, _lp], C.c_int),
    "regc_set_walker_ne": ([_h, C.c_int, C.c_int, _ip, _ip, _lp], C.c_int),
    "regc_cycle": ([_h, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "regc_cycle_traced": ([_h, C.c_int, C.c_double, C.c_int, C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "regc_cycle_md": ([_h, C.c_int, C.c_double, C.c_int, C.c_float, C.c_float, C.POINTER(C.c_int)], C.c_int),
    "regc_md": ([_h, C.c_int, C.c_float, C.c_float, _fp], C.c_int),
    "regc_histograms": ([_h, _lp, _lp, _lp, _dp, _lp], C.c_int),
    "regc_reset_histograms": ([_h], C.c_int),
    "regc_set_state_windows": ([_h, C.c_int, C.c_double, _dp], C.c_int),
    "regc_state_histograms": ([_h, _lp, _dp, _dp], C.c_int),
    "regc_free": ([_h], None),
    "regc_set_walkers": ([_h, _fp, _ip, _ip], C.c_int),
    "regc_set_cluster": ([_h, C.c_int, C.c_int], C.c_int),
    "regc_checkpoint": ([_h, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
    "regc_restore": ([_h, C.c_void_p, C.c_size_t], C.c_int),
    "regc_get_walkers": ([_h, _fp, _ip, _dp, _ip], C.c_int),
    "regc_check_energy": ([_h, _dp], C.c_int),
    "regc_counters": ([_h, _lp, _lp, _lp], C.c_int),
    "regc_warps_per_walker": ([_h, C.POINTER(C.c_int)], C.c_int),
    "regc_structure_init": ([_h, C.c_void_p], C.c_int),
    "regc_structure_sample": ([_h], C.c_int),
    "regc_structure_count": ([_h, C.POINTER(C.c_int64)], C.c_int),
    "regc_structure_reset": ([_h], C.c_int),
    "regc_structure_timing": ([_h, _dp, _dp, _dp, _dp], C.c_int),
    "regc_aiat": ([_h, C.c_int, _dp, _dp, _dp, C.c_void_p], C.c_int),
    "regc_mu_of_pressure": ([C.c_int, _dp, _dp, C.c_double, _dp], C.c_int),
    "regc_pressure_of_mu": ([C.c_int, _dp, _dp, C.c_double, _dp], C.c_int),
    "regc_aiat_config": ([_h, C.c_int, _fp, C.POINTER(C.c_int32)], C.c_int),
    "regc_structure_get": ([_h, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p], C.c_int),
    "regc_structure_reweight": ([_h, C.c_int, _dp, _dp, C.c_int, C.c_int, C.c_double, C.c_int, _dp, _dp, _dp,
                                 _dp, C.POINTER(C.c_int)], C.c_int),
    "regc_reweight": ([_h, C.c_int, _dp, _dp, C.c_double, C.c_int, _dp, _dp, _dp, _ip], C.c_int),
    "regc_reweight2": ([_h, C.c_int, _dp, _dp, _dp, C.c_double, C.c_int, _dp, _dp, _dp, _dp, _dp, _ip], C.c_int),
    "regc_mbar_last_info": ([C.POINTER(MbarInfo)], C.c_int),
    "regc_test_expire_waits": ([_h], C.c_int),
    "regc_mbar_solve": ([C.c_int, _dp, _dp, C.c_double, _dp, C.c_int, _ip, _dp, _dp, C.c_double,
                         C.c_int, _dp, _dp, _ip, C.c_void_p], C.c_int),
    "regc_mbar_solve_static": ([C.c_int, _dp, _dp, C.c_double, _dp, C.c_int, _ip, _dp, _dp, C.c_double,
                                C.c_int, _dp, _dp, _ip, C.c_void_p], C.c_int),
    "regc_mbar_query": ([C.c_int, _dp, _dp, C.c_double, C.c_int, _ip, _dp, _dp, _dp, C.c_int,
                         _dp, _dp, _dp, C.c_void_p], C.c_int),
    "regc_surrogate_set": ([_h, _fp], C.c_int),
    "regc_surrogate_get": ([_h, _fp], C.c_int),
    "regc_surrogate_init": ([_h, C.c_uint64, C.c_float], C.c_int),
    "regc_set_mode": ([_h, C.c_int], C.c_int),
    "regc_surrogate_eval": ([_h, C.c_int, C.c_int, _fp, _fp, _fp], C.c_int),
    "regc_surrogate_harvest": ([_h, C.c_int, C.c_int, C.c_float, C.c_int, _lp], C.c_int),
    "regc_surrogate_dataset": ([_h, C.c_int64, _fp, _fp, _lp], C.c_int),
    "regc_surrogate_train": ([_h, C.c_int, C.c_int, C.c_float, _fp], C.c_int),
    "regc_surrogate_gradient": ([C.c_int, _fp, _fp, _fp, _fp, _fp, C.c_void_p], C.c_int),
    "regc_surrogate_gradient_bf16": ([C.c_int, _fp, _fp, _fp, _fp, _fp, C.c_void_p], C.c_int),
    "regc_surrogate_set_dataset": ([_h, C.c_int64, _fp, _fp, C.c_int], C.c_int),
    "regc_batch_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "regc_batch_run": ([_h, C.c_int], C.c_int),
    "regc_batch_autotune": ([_h, C.c_int], C.c_int),
    "regc_batch_plan": ([_h, C.c_int, C.POINTER(C.c_int), _ip, _ip, _ip, _ip, _ip, _dp], C.c_int),
    "regc_batch_sync": ([_h], C.c_int),
    "regc_batch_free": ([_h], None),
    "regc_status_string": ([C.c_int], C.c_char_p),
}

SURROGATE_PARAMS = 5313

_lib = None


def declared_symbols(header: str = HEADER):
    """Entry points declared in include/regc.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(regc_[a-z0-9_]+)\s*\(", text)))


def lib():
    """The loaded library (raises if it has not been built or cannot load)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libregc.so is not built (run paper_1908_11118_gb300/build.py or "
                               "__graft_entry__.build()); there is no fallback implementation")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != REGC_OK:
        raise RegcError(status, where)
