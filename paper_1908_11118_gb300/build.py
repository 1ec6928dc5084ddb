"""Build the REGC CUDA library in-tree: paper_1908_11118_gb300/_build/libregc.so
(and libregc_probe.so, the FP32 peak probe the benchmark quotes its roofline
against).

Each translation unit is compiled for sm_103a only, in parallel, then linked
into one shared library exporting the C ABI of include/regc.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libregc.so")
# measurement tooling (the FP32 peak probe), kept out of the library proper
PROBE_LIB = os.path.join(BUILD, "libregc_probe.so")
PROBE_SOURCES = ["probe.cu"]
SOURCES = ["sweep.cu", "exchange.cu", "mbar.cu", "regc_api.cu", "mbar_static.cu", "surrogate.cu", "walkers.cu", "batch.cu", "md.cu", "structure.cu"]
HEADERS = ["regc_internal.cuh", "launch.h", "mbar.h", "surrogate.cuh", "handle.h", "cells.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--ptxas-options=-v" if os.environ.get("REGC_PTXAS_VERBOSE") else "-w"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the REGC library needs the CUDA toolkit to build")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    inc = os.path.join(os.path.dirname(HERE), "include")
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(inc, "regc.h"),
                                                        os.path.join(inc, "regc_probe.h"), __file__]
    objs = []
    jobs = []
    probe_objs = [os.path.join(BUILD, src.replace(".cu", ".o")) for src in PROBE_SOURCES]
    for src in SOURCES + PROBE_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if src in SOURCES:
            objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc(), *ARCH, *FLAGS, "-I", inc, "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s" % cmd[-3])
    for lib, lobjs in ((LIB, objs), (PROBE_LIB, probe_objs)):
        if force or jobs or _stale(lib, lobjs):
            tmp = lib + ".tmp%d" % os.getpid()
            r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *lobjs], capture_output=True, text=True)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("linking %s failed" % os.path.basename(lib))
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
