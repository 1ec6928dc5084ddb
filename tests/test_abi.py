"""The C-ABI library builds, loads and exports every declared entry point.

These tests make no compute call: they run on a machine without a GPU.  The
argument checks of regc_init_grid happen before any CUDA call, so invalid
problem statements are rejected here too.
"""
import ctypes as C
import os

import numpy as np
import pytest

import workloads as W
from paper_1908_11118_gb300 import _lib
from paper_1908_11118_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing
    assert set(_lib.SIGNATURES) == set(names)


def test_probe_library_exports_its_header():
    """The FP32 peak probe (measurement tooling) is its own library: it
    exports what include/regc_probe.h declares, and libregc.so does not."""
    B.build()
    probe = C.CDLL(B.PROBE_LIB)
    names = _lib.declared_symbols(os.path.join(os.path.dirname(_lib.HEADER), "regc_probe.h"))
    assert names == ["regc_probe_fp32_peak"]
    assert all(hasattr(probe, n) for n in names)
    assert not hasattr(_lib.lib(), "regc_probe_fp32_peak")


def test_status_strings(lib):
    assert lib.regc_status_string(0) == b"ok"
    assert lib.regc_status_string(-1) == b"invalid argument"
    assert lib.regc_status_string(-5) == b"cell-list capacity exceeded"


def _structs(p):
    pot = _lib.Potential()
    pot.n_types = p.n_types
    for i in range(4):
        for j in range(4):
            pot.eps[i][j] = p.eps[i][j]
            pot.sigma[i][j] = p.sigma[i][j]
    pot.rc = p.rc
    xyz = np.ascontiguousarray(p.surf_xyz, np.float32)
    typ = np.ascontiguousarray(p.surf_type, np.int32)
    surf = _lib.Surface(len(typ), xyz.ctypes.data_as(C.POINTER(C.c_float)),
                        typ.ctypes.data_as(C.POINTER(C.c_int32)), p.Lx, p.Ly, p.Lz, p.periodic_z,
                        p.z_lo, p.z_hi)
    kT = np.ascontiguousarray(p.kT, np.float64)
    mu = np.ascontiguousarray(p.mu, np.float64)
    grid = _lib.GridSpec(len(kT), len(mu), kT.ctypes.data_as(C.POINTER(C.c_double)),
                         mu.ctypes.data_as(C.POINTER(C.c_double)), p.lambda0, p.nmax,
                         p.moves_per_sweep, p.max_disp, p.p_disp, p.e_lo, p.e_bin, p.n_e_bins)
    return pot, surf, grid, (xyz, typ, kT, mu)


@pytest.mark.parametrize("bad", [
    dict(rc=0.0), dict(Lx=4.0), dict(nmax=0), dict(nmax=5000), dict(moves_per_sweep=0),
    dict(p_disp=1.5), dict(kT=np.array([0.6, -1.0])), dict(e_bin=0.0), dict(lambda0=0.0),
    dict(z_hi=1.0), dict(surf_type=np.full(32, 3, np.int32)), dict(periodic_z=1),
])
def test_init_rejects_invalid_problems(lib, bad):
    p = W.fcc100_small().replace(**bad)
    pot, surf, grid, keep = _structs(p)
    h = C.c_void_p(123)
    st = lib.regc_init_grid(C.byref(pot), C.byref(surf), C.byref(grid), 0, None, C.byref(h))
    assert st == -1
    assert not h.value


def test_null_handles_are_rejected(lib):
    assert lib.regc_sweep(None, 1) == -1
    assert lib.regc_exchange(None) == -1
    assert lib.regc_check_energy(None, None) == -1
    lib.regc_free(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        _lib.lib()


def test_move_record_layout_matches_header(tmp_path):
    """The binding's trace dtype has the size and field offsets of the C struct."""
    import subprocess
    from paper_1908_11118_gb300.regc import MOVE_DTYPE
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    fields = MOVE_DTYPE.names
    src = tmp_path / "layout.c"
    body = "".join('printf("%%zu\\n", offsetof(regc_move_record, %s));\n' % f for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "regc.h"\nint main(void){\n'
                   'printf("%zu\\n", sizeof(regc_move_record));\n' + body + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == MOVE_DTYPE.itemsize
    assert out[1:] == [MOVE_DTYPE.fields[f][1] for f in fields]


def test_batch_argument_checks_without_gpu(lib):
    out = C.c_void_p(123)
    arr = (C.c_void_p * 1)(None)
    assert lib.regc_batch_create(arr, 0, 10, None, C.byref(out)) == -1 and not out.value
    assert lib.regc_batch_create(arr, 1, 10, None, C.byref(out)) == -1 and not out.value
    assert lib.regc_batch_create(None, 1, 10, None, C.byref(out)) == -1
    assert lib.regc_batch_run(None, 1) == -1
    assert lib.regc_batch_sync(None) == -1
    lib.regc_batch_free(None)
