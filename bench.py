#!/usr/bin/env python3
"""Benchmark: GCMC trial moves/s over all replicas of the REGC sampler.

Workload (the paper-scale LJ surface-gas system): frozen fcc(111) slab of
12x12x4 atoms, gas region 12 high, eps_sg = 2, 32 kT x 32 mu = 1024 replicas,
Nmax 512, 20 trial moves per sweep.  Initial walkers: N ~ U{0..256} particles
on a jittered lattice (seeded), then untimed equilibration sweeps.

One step = 10 sweeps of every replica (one sweep-kernel launch) followed by one
collective replica-exchange attempt (one exchange-kernel launch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]

own arm: device-timed (CUDA events on the library's stream) steps, with the L2
flushed (256 MB memset) before every timed step; the JSON line adds the
FP32-ALU roofline of the sweep kernel, the end-to-end rate through the C ABI
with host buffers, sampled SM clocks, and the FP64 CPU oracle timed on a
bounded sample on the host cores.
reference arm: the FP64 CPU oracle on the same workload and metric.
Under torchrun (N > 1) every rank runs its own independent 1024-replica grid
(seed = rank): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import ctypes
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

SWEEPS_PER_STEP = 10
# DRAM bytes (read + write) of one sweep-kernel launch on the benchmark
# workload from an ncu capture of the current kernel
# (dram__bytes_read.sum 4336384 + dram__bytes_write.sum 0); None whenever the
# kernel has changed since its last capture
SWEEP_TRAFFIC_BYTES = 4336384 + 0
FLOPS_PER_PAIR = 20            # dx,dy,dz 3, xy minimum image 4, r^2 5, r^-2 1, s^6 3, 4eps s^6(s^6-1) 4
SM_COUNT, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0
METRIC = "GCMC trial moves/s over all replicas"
DA_SMALL = ("fcc100 4x4x2 slab in a 6.25 x 6.25 x 10 box (hard wall at the top), 4 kT x 4 mu = 16 "
            "replicas, Nmax 32, 20 moves/sweep; step = 10 sweeps + 1 replica-exchange attempt")
WORKLOAD = ("fcc111 12x12x4 slab + LJ gas, 32 kT x 32 mu = 1024 replicas, Nmax 512, "
            "20 moves/sweep; step = 10 sweeps + 1 replica-exchange attempt")


def bench_config(args):
    """The `config` of the headline line, identical in both arms: the same
    workload, the same seeded start and the same equilibration protocol."""
    return {"workload": WORKLOAD, "equilibration_sweeps": args.equil,
            "start": "seeded lattice state (seed 0), then the equilibration sweeps untimed",
            "l2": "GPU arm: flushed (256 MB memset) before every timed step; host arm: n/a"}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--equil", type=int, default=500, help="untimed equilibration sweeps")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--da", type=int, default=1, help="1: add the plain vs delayed-acceptance comparison")
    ap.add_argument("--batch", type=int, default=1, help="1: add the batched uneven workload")
    ap.add_argument("--md", type=int, default=1, help="1: add MD segments (REGCMD) of the main workload")
    ap.add_argument("--md-segments", type=int, default=10)
    ap.add_argument("--cluster", type=int, default=1, help="1: add the cluster-in-gas workload")
    ap.add_argument("--paper-cycle", type=int, default=1,
                    help="1: add the paper's LJ run through the REGC cycle (x0 = 0.99)")
    ap.add_argument("--paper-steps", type=int, default=120000, help="REGC steps of that run")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--production", type=int, default=100000,
                    help="sweeps of the 1024-replica production run reweighted to <N>(T, p) (0: skip)")
    ap.add_argument("--two-species", type=int, default=1, help="1: add the two-species workload")
    ap.add_argument("--two-species-steps", type=int, default=20)
    ap.add_argument("--two-species-sweeps", type=int, default=100000)
    ap.add_argument("--cluster-production", type=int, default=20000,
                    help="sweeps of configuration 5 with the surrogate in a batch (0: skip; 1e6 is the full run)")
    ap.add_argument("--da-train-steps", type=int, default=3000)
    ap.add_argument("--da-steps-small", type=int, default=1000)
    ap.add_argument("--da-steps-large", type=int, default=60)
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def combine_rank_results(times_ms, moves_per_rank):
    """Whole-job throughput: units of all ranks / the slowest rank's time."""
    t = max(times_ms)
    return sum(moves_per_rank) / (t / 1e3), t


def job_throughput(local_ms, local_moves, world, device):
    """Whole-job throughput across the process group: every rank contributes
    its moves and timed milliseconds; the job time is the slowest rank's.
    Returns (moves/s over all ranks, max ms)."""
    if world == 1:
        return combine_rank_results([local_ms], [local_moves])
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    m = torch.tensor([float(local_moves)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    tmax = float(t.item())
    return float(m.item()) / (tmax / 1e3), tmax


def fp32_peak(stream=None):
    """FP32 ALU peak: the peaks file's, if it has one; else measured here by the
    FFMA-loop probe (libregc_probe.so, include/regc_probe.h); the unit-count
    figure is printed beside it."""
    derived = SM_COUNT * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("fp32_tflops", "fp32_tflops_sustained"):
                if k in d:
                    return float(d[k]), "MEASURED_PEAKS.json (%s)" % k
        except Exception:
            pass
    from paper_1908_11118_gb300 import build as B
    probe = ctypes.CDLL(B.PROBE_LIB)
    probe.regc_probe_fp32_peak.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    probe.regc_probe_fp32_peak.restype = ctypes.c_int
    from paper_1908_11118_gb300.regc import _stream_handle
    handle = _stream_handle(stream)

    def once():
        t = ctypes.c_double(0.0)
        rc = probe.regc_probe_fp32_peak(20000, handle, ctypes.byref(t))
        if rc != 0:
            raise RuntimeError("regc_probe_fp32_peak returned %d" % rc)
        return t.value
    best = max(once() for _ in range(3))
    return best, ("measured on this GPU: FFMA-loop probe (regc_probe_fp32_peak, best of 3); unit-count figure "
                  "152 SMs x 128 lanes x 2 flop x 2070 MHz = %.1f TFLOP/s" % derived)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = [r.split(",") for r in open(self.file.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) > 8
                          for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def initial_state(p, seed):
    rng = np.random.default_rng(seed)
    n0 = rng.integers(0, p.nmax // 2 + 1, p.S)
    return W.lattice_walkers(p, n0, seed=seed)


# ------------------------------------------------------------- CPU oracle

def time_oracle(p, pos, n, seconds, min_steps=1, max_steps=None, warmup=0, threads=0, equil=0, orc=None):
    """Run the FP64 oracle on the workload in steps of 10 sweeps + exchange
    until `seconds` have passed, after `equil` untimed equilibration sweeps
    (the GPU arm's protocol) unless an equilibrated oracle `orc` is given.
    Returns (moves/s, steps timed, seconds, threads used, oracle)."""
    from oracle import oracle as O
    O.build()
    if orc is None:
        orc = O.Oracle(p, pos=pos, n=n, n_threads=threads)
        if equil > 0:
            orc.run(equil, exchange_every=SWEEPS_PER_STEP, hist=False)
    orc.n_threads = threads
    for _ in range(warmup):
        orc.run(SWEEPS_PER_STEP, exchange_every=SWEEPS_PER_STEP, hist=True)
    steps, t0 = 0, time.perf_counter()
    while True:
        orc.run(SWEEPS_PER_STEP, exchange_every=SWEEPS_PER_STEP, hist=True)
        steps += 1
        el = time.perf_counter() - t0
        if (el >= seconds and steps >= min_steps) or (max_steps and steps >= max_steps):
            break
    moves = steps * p.S * SWEEPS_PER_STEP * p.moves_per_sweep
    return moves / el, steps, el, (threads if threads > 0 else os.cpu_count()), orc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    p = W.fcc111_paper_scale(seed=0)
    pos, n = initial_state(p, 0)
    rate, steps, el, cores, _ = time_oracle(p, pos, n, seconds=0.0, min_steps=args.steps,
                                            max_steps=args.steps, warmup=args.warmup,
                                            equil=args.equil)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "moves/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": el / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(args),
        "cpu_baseline": {"value": rate, "unit": "moves/s", "cores": cores, "kind": "oracle",
                         "sample": "full 1024-replica workload, %d steps of 10 sweeps + exchange" % steps},
        "e2e": {"value": rate, "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------- delayed acceptance arm

DA_ROWS_PER_WALKER = (8, 8)     # particle rows, probe rows per walker per harvest
DA_CLIP = 8.0                   # training targets clipped from above (eps units)


def timed_run(g, torch, stream, flush, steps, n_batches):
    """steps of (10 sweeps + exchange), device-timed per step with the L2
    flushed before each; batch means of <N> per state.  Returns
    (seconds, trial moves, accepted moves, pair counters delta, per-state
    batch-mean <N> [n_batches, S])."""
    g.reset_histograms()
    nv = np.arange(g.nmax + 1)
    per = max(1, steps // n_batches)
    ev = []
    nb = []
    prev = g.histograms()["hN"]
    for k in range(per * n_batches):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.sweep(SWEEPS_PER_STEP)
        g.exchange()
        e1.record(stream)
        ev.append((e0, e1))
        if (k + 1) % per == 0:
            h = g.histograms()["hN"]
            d = h - prev
            prev = h
            nb.append((d @ nv) / np.maximum(d.sum(axis=1), 1))
    torch.cuda.synchronize()
    secs = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    mv, _, pr = g.counters()
    return secs, int(mv[:, :, 0].sum()), int(mv[:, :, 1].sum()), pr, np.array(nb)


def harvest_and_train(g, p, torch, rows_target, train_steps, seed=0):
    """The surrogate of a handle: initialised from the seed, 200 plain sweeps,
    then rows harvested every 10 sweeps until rows_target, then train_steps
    Adam steps on 1024-row mini-batches."""
    g.surrogate_init(seed=seed, scale=1.0)
    g.run(200, exchange_every=SWEEPS_PER_STEP)
    per = p.S * sum(DA_ROWS_PER_WALKER)
    harvests = max(1, -(-rows_target // per))
    t0 = time.perf_counter()
    rows = 0
    for _ in range(harvests):
        g.sweep(SWEEPS_PER_STEP)
        g.exchange()
        rows = g.surrogate_harvest(*DA_ROWS_PER_WALKER, DA_CLIP, capacity=harvests * per)
    torch.cuda.synchronize()
    t_harvest = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = g.surrogate_train(train_steps, 1024, 1e-3)
    t_train = time.perf_counter() - t0
    return {"rows": rows, "harvests": harvests, "rows_per_walker_per_harvest": list(DA_ROWS_PER_WALKER),
            "target_clip": DA_CLIP, "steps": train_steps, "batch": 1024, "lr": 1e-3,
            "loss_first": float(np.mean(loss[:20])), "loss_last": float(np.mean(loss[-100:])),
            "harvest_s": t_harvest, "train_s": t_train}


def delayed_acceptance_arm(p, name, torch, stream, flush, rows_target, train_steps, timed_steps, seed=0):
    """Train the surrogate on rows the plain sampler generates, then time the
    plain and the delayed-acceptance sweep from the same state."""
    from paper_1908_11118_gb300 import Regc

    rng = np.random.default_rng(seed)
    if p.n_cluster:
        pos0, n0 = W.cluster_initial(p, rng.integers(0, (p.nmax - p.n_cluster) // 2 + 1, p.S), seed=seed)
    else:
        pos0, n0 = W.lattice_walkers(p, rng.integers(0, p.nmax // 2 + 1, p.S), seed=seed)
    g = Regc(p, stream=stream)
    g.set_walkers(pos0, n0)
    training = harvest_and_train(g, p, torch, rows_target, train_steps, seed)
    state = g.get_walkers()
    res, se_of, mean_of = {}, {}, {}
    for mode in ("plain", "delayed"):
        g.set_walkers(state[0], state[1], state[3])
        g.set_mode(mode == "delayed")
        g.run(50, exchange_every=SWEEPS_PER_STEP)
        secs, trials, acc, pr, nb = timed_run(g, torch, stream, flush, timed_steps, 20)
        se = nb.std(axis=0, ddof=1) / np.sqrt(len(nb))
        se_of[mode], mean_of[mode] = se, nb.mean(axis=0)
        exact = int(pr[5]) if mode == "delayed" else int(pr[3])
        res[mode] = {"trial_moves_per_s": trials / secs, "accepted_moves_per_s": acc / secs,
                     "acceptance": acc / trials, "exact_evaluations_per_accepted_move": exact / max(acc, 1),
                     "screen_pass_fraction": (int(pr[5]) / max(int(pr[4]), 1)) if mode == "delayed" else None,
                     "mean_N_stderr": float(np.mean(se)), "seconds": secs, "trial_moves": trials}
    g.set_mode(False)
    g.close()
    pl, da = res["plain"], res["delayed"]
    # efficiency per state: eta = 1 / (stderr(<N>)^2 x time); states whose N
    # never moved (stderr 0) carry no information and are left out
    sp, sd = np.asarray(se_of["plain"]), np.asarray(se_of["delayed"])
    ok = (sp > 0) & (sd > 0)
    ratio = (sp[ok] ** 2 * pl["seconds"]) / (sd[ok] ** 2 * da["seconds"])
    # time for every state's stderr to reach 0.02 max(1, <N>)
    for mode, se in se_of.items():
        tgt = 0.02 * np.maximum(1.0, mean_of[mode])
        res[mode]["seconds_to_stderr_2pct_all_states"] = float(res[mode]["seconds"] * np.max((se / tgt) ** 2))
    return {
        "workload": name,
        "training": training,
        "plain": pl, "delayed": da,
        "trial_moves_ratio": da["trial_moves_per_s"] / pl["trial_moves_per_s"],
        "accepted_moves_ratio": da["accepted_moves_per_s"] / pl["accepted_moves_per_s"],
        "eta_ratio_median": float(np.median(ratio)) if ratio.size else None,
        "eta_ratio_worst": float(np.min(ratio)) if ratio.size else None,
        "eta_states": int(ratio.size),
        "timed_steps": timed_steps,
    }


# ------------------------------------------------------ batched uneven arm

CLUSTER_WORKLOAD = ("15 sigma periodic cube, A4 cluster (eps_AA 4, sigma_AA 1.1; displacement only) in a B gas "
                    "(eps_BB 0.5, eps_AB 2, sigma 1; grand-canonical), 64 kT x 64 mu = 4096 replicas, Nmax_B 64; "
                    "step = 10 sweeps + 1 replica-exchange attempt")
BATCH_WORKLOAD = ("256 systems x (4 kT x 4 mu) = 4096 replicas; 3-layer fcc(100) slabs of nx x ny atoms, "
                  "nx, ny ~ U{6..16}; gas 8-16 high; Nmax = 2^k, k ~ U{6..11}; N0 ~ U{0..Nmax/2} capped at "
                  "90% of a 1.1-spacing lattice; step = 10 sweeps + 1 exchange attempt per system")


def cluster_production_arm(torch, stream, sweeps, rows_target, train_steps, equil=500, seed=0):
    """Configuration 5's production: the 4096-replica cluster-in-gas grid
    sampled with the trained surrogate (delayed acceptance) through a batch
    (the persistent delayed-acceptance kernel in a captured graph, shape
    autotuned), `sweeps` sweeps with per-state energy windows (KS check of
    the two halves, Sec. III.A), then the pooled (N_B, E) histogram reweighted
    in FP64 (Sec. II.B) to <N_B> on a (T, p) grid (mu from p by the ideal-gas
    reservoir of Sec. III.A)."""
    from paper_1908_11118_gb300 import Batch, Regc, mu_of_pressure

    p = W.cluster_in_gas(seed=seed)
    rng = np.random.default_rng(seed)
    pos0, n0 = W.cluster_initial(p, rng.integers(0, (p.nmax - p.n_cluster) // 2 + 1, p.S), seed=seed)
    g = Regc(p, stream=stream)
    g.set_walkers(pos0, n0)
    training = harvest_and_train(g, p, torch, rows_target, train_steps, seed)
    g.set_mode(True)
    g.run(equil, exchange_every=SWEEPS_PER_STEP)
    bt = Batch([g], sweeps_per_step=SWEEPS_PER_STEP, stream=stream)
    bt.autotune(3)   # each shape timed three times, the fastest kept
    plan = bt.plan()
    g.set_state_windows(1024, 0.25, None)
    g.reset_histograms()
    mv0 = g.counters()
    torch.cuda.synchronize()
    steps = max(2, sweeps // SWEEPS_PER_STEP)
    chunk = 100
    half = None
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        bt.run(k)
        done += k
        if half is None and done >= steps // 2:
            bt.sync()
            half = g.state_histograms()[0]
    bt.sync()
    run_s = time.perf_counter() - t0
    full = g.state_histograms()[0]
    bt.close()
    mv1 = g.counters()
    ks, crit = ks_halves(half, full - half)
    h = g.histograms()
    kT_q = np.geomspace(0.6, 1.5, 12)
    kT_mid = float(np.sqrt(0.6 * 1.5))
    p_lo, p_hi = (kT_mid * np.exp(np.array([-6.0, -2.0]) / kT_mid) / (p.lambda0 / np.sqrt(kT_mid)) ** 3)
    p_q = np.geomspace(p_lo, p_hi, 12)
    T, P = np.meshgrid(kT_q, p_q, indexing="ij")
    mu_q = mu_of_pressure(T.ravel(), P.ravel(), p.lambda0)
    t1 = time.perf_counter()
    nm, pN, f, iters = g.reweight(T.ravel(), mu_q, tol=1e-9, max_iter=200000)
    rw_s = time.perf_counter() - t1
    mbar = mbar_summary()
    trials = int((mv1[0][:, :, 0] - mv0[0][:, :, 0]).sum())
    screened = int(mv1[2][4] - mv0[2][4])
    passed = int(mv1[2][5] - mv0[2][5])
    g.set_mode(False)
    g.close()
    return {"workload": CLUSTER_WORKLOAD, "sampler": "delayed acceptance (trained surrogate) in a batch",
            "training": training, "equilibration_sweeps": equil, "sweeps": steps * SWEEPS_PER_STEP,
            "batch_plan": plan, "run_s": run_s, "trial_moves_per_s": trials / run_s,
            "screen_pass_fraction": passed / max(screened, 1),
            "observations": int(h["omega"].sum()), "pooled_bins_occupied": int(np.count_nonzero(h["hNE"])),
            "e_out": int(h["e_out"].sum()),
            "convergence_ks_halves": {"median": float(np.median(ks)), "max": float(np.max(ks)),
                                      "states_unchanged_at_1pct": int(np.sum(ks < crit))},
            "reweight_s": rw_s, "mbar_iterations": iters, "mbar": mbar,
            "phase_map": {"kT": kT_q.tolist(), "p": p_q.tolist(),
                          "N_B_mean": nm.reshape(12, 12).round(3).tolist(),
                          "N_B_most_probable": np.argmax(pN, axis=1).reshape(12, 12).tolist()}}


def batched_uneven_arm(torch, steps, seed=0):
    """The batched uneven workload: every system's walkers in size-class
    persistent kernels of one captured graph (autotuned), against the same
    systems stepped one handle at a time."""
    from paper_1908_11118_gb300 import Batch, Regc

    ps = W.uneven_batch(256, seed=seed)
    t0 = time.perf_counter()
    hs = []
    for i, p in enumerate(ps):
        pos, n = W.uneven_initial(p, seed * 7919 + i)
        h = Regc(p)
        h.set_walkers(pos, n)
        hs.append(h)
    t_setup = time.perf_counter() - t0
    S = sum(p.S for p in ps)
    moves_per_step = S * SWEEPS_PER_STEP * 20
    stream = torch.cuda.Stream()
    bt = Batch(hs, sweeps_per_step=SWEEPS_PER_STEP, stream=stream)
    plan_default = bt.plan()
    t0 = time.perf_counter()
    bt.autotune(3)   # each shape timed three times, the fastest kept
    t_tune = time.perf_counter() - t0
    bt.run(3)                                   # warm-up (captures the graph)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bt.run(1)
        b.record(stream)
        ev.append((a, b))
    bt.sync()
    batched_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    # the same systems, one handle after another on one stream (a fixed number of steps)
    k1 = max(2, steps // 5)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(k1):
        for h in hs:
            h.sweep(SWEEPS_PER_STEP)
            h.exchange()
    b.record()
    torch.cuda.synchronize()
    single_s = a.elapsed_time(b) / 1e3
    drift = max(h.check_energy() for h in hs)
    acc = sum(int(h.counters()[0][:, :, 1].sum()) for h in hs)
    trials = sum(int(h.counters()[0][:, :, 0].sum()) for h in hs)
    out = {
        "workload": BATCH_WORKLOAD,
        "replicas": S,
        "nmax_classes": sorted({p.nmax for p in ps}),
        "trial_moves_per_s": moves_per_step * steps / batched_s,
        "ms_per_step": batched_s / steps * 1e3,
        "one_handle_at_a_time_moves_per_s": moves_per_step * k1 / single_s,
        "acceptance": acc / max(trials, 1),
        "plan_default": plan_default,
        "plan_tuned": bt.plan(),
        "setup_s": t_setup,
        "autotune_s": t_tune,
        "energy_drift_max": drift,
        "timed_steps": steps,
        "l2": "flushed (256 MB memset) before every timed step",
    }
    bt.close()
    for h in hs:
        h.close()
    return out


# ---------------------------------------------------------------- REGCMD

def regcmd_arm(g, p, torch, stream, flush, segments, n_steps=10, dt=0.005, tau=0.1):
    """MD segments of every walker of the benchmark workload (regc_md) from its
    current state, device-timed per segment with the L2 flushed before each;
    and REGCMD steps (regc_cycle_md: the x0 choice of Sec. II.A, then one MD
    segment)."""
    n_mean = float(np.mean(g.get_walkers()[1]))
    for _ in range(2):
        g.md(n_steps, dt, tau, kinetic=False)
    ev = []
    for _ in range(segments):
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.md(n_steps, dt, tau, kinetic=False)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    seg_ms = sum(a.elapsed_time(b) for a, b in ev) / segments
    ev = []
    for _ in range(segments):
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.cycle_md(1, 0.99, n_steps, dt, tau)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    cyc_ms = sum(a.elapsed_time(b) for a, b in ev) / segments
    drift = g.check_energy()
    return {
        "workload": WORKLOAD,
        "segment": {"steps": n_steps, "dt": dt, "tau": tau},
        "mean_N": n_mean,
        "ms_per_segment": seg_ms,
        "particle_steps_per_s": p.S * n_mean * n_steps / (seg_ms / 1e3),
        "ms_per_cycle": cyc_ms,
        "cycle": "one REGCMD step (regc_cycle_md, x0 = 0.99): a particle-exchange attempt per replica or a "
                 "replica-exchange attempt, then one MD segment",
        "energy_drift": drift,
        "timed_segments": segments,
    }


# ---------------------------------------------------------------- the paper's LJ run

PAPER_CYCLE = ("the paper's LJ surface system (Sec. III.A) in eV and Angstrom, in its own cell: the 3x3 "
               "hexagonal supercell of a two-layer fcc(111) A slab (A18, lattice vectors 11.489 A at 60 deg) "
               "under B gas in a 48 A zone, 10 T (200-650 K) x 16 mu (-2.4..-0.9 eV) = 160 replicas, "
               "Nmax 160; REGC cycle x0 = 0.99, 10 displacements per step")


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) from the peaks file, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return float(json.load(open(path))["hbm_gbs"]), "MEASURED_PEAKS.json (hbm_gbs)"
        except Exception:
            pass
    return 6800.0, "fallback 6.8 TB/s"


def ks_halves(h1, h2):
    """Per row: the two-sample Kolmogorov-Smirnov distance between the
    histograms h1 and h2 (same bins), and its 1 % critical value."""
    c1 = np.cumsum(h1, axis=1) / np.maximum(h1.sum(axis=1, keepdims=True), 1)
    c2 = np.cumsum(h2, axis=1) / np.maximum(h2.sum(axis=1, keepdims=True), 1)
    n1, n2 = np.maximum(h1.sum(axis=1), 1), np.maximum(h2.sum(axis=1), 1)
    return np.max(np.abs(c1 - c2), axis=1), 1.63 * np.sqrt((n1 + n2) / (n1 * n2))


def production_arm(torch, stream, sweeps, equil=2000, seed=0):
    """Configuration 2's production run: the 1024-replica workload for
    `sweeps` sweeps after `equil` equilibration sweeps, each state's energies
    in a window of its own (centred on its mean after equilibration), then the
    pooled (N, E) histogram reweighted in FP64 (Sec. II.B) to <N> and the most
    probable N on a (T, p) grid (mu from p by the ideal-gas reservoir of
    Sec. III.A).  The convergence check of Sec. III.A compares each state's
    energy distribution between the two halves of the run."""
    from paper_1908_11118_gb300 import Regc, mu_of_pressure

    p = W.fcc111_paper_scale(seed=seed)
    pos, n = initial_state(p, seed)
    g = Regc(p, stream=stream)
    g.set_walkers(pos, n)
    g.run(equil, exchange_every=SWEEPS_PER_STEP)
    g.set_state_windows(1024, 0.5, None)
    g.reset_histograms()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    half = None
    chunk = 1000
    done = 0
    while done < sweeps:
        g.run(min(chunk, sweeps - done), exchange_every=SWEEPS_PER_STEP)
        done += min(chunk, sweeps - done)
        if half is None and done >= sweeps // 2:
            half = g.state_histograms()[0]
    full = g.state_histograms()[0]
    torch.cuda.synchronize()
    run_s = time.perf_counter() - t0
    ks, crit = ks_halves(half, full - half)
    h = g.histograms()
    # (T, p) query grid: 12 temperatures over the grid's range, 12 pressures
    # spanning mu -6 .. -2 at the middle temperature
    kT_q = np.geomspace(0.6, 1.5, 12)
    kT_mid = float(np.sqrt(0.6 * 1.5))
    p_lo, p_hi = (kT_mid * np.exp(np.array([-6.0, -2.0]) / kT_mid) / (p.lambda0 / np.sqrt(kT_mid)) ** 3)
    p_q = np.geomspace(p_lo, p_hi, 12)
    T, P = np.meshgrid(kT_q, p_q, indexing="ij")
    mu_q = mu_of_pressure(T.ravel(), P.ravel(), p.lambda0)
    t1 = time.perf_counter()
    nm, pN, f, iters = g.reweight(T.ravel(), mu_q, tol=1e-9, max_iter=200000)
    rw_s = time.perf_counter() - t1
    mbar = mbar_summary()
    g.close()
    return {"workload": WORKLOAD, "sweeps": sweeps, "equilibration_sweeps": equil,
            "run_s": run_s, "trial_moves_per_s": p.S * sweeps * p.moves_per_sweep / run_s,
            "observations": int(h["omega"].sum()), "pooled_bins_occupied": int(np.count_nonzero(h["hNE"])),
            "e_out": int(h["e_out"].sum()),
            "state_windows": {"bins": 1024, "e_bin": 0.5,
                              "outside": int(full[:, 0].sum() + full[:, -1].sum())},
            "convergence_ks_halves": {"median": float(np.median(ks)), "max": float(np.max(ks)),
                                      "states_unchanged_at_1pct": int(np.sum(ks < crit)),
                                      "note": "per-state energy histograms of the two halves; samples "
                                              "one sweep apart are correlated, so the critical value "
                                              "is optimistic"},
            "reweight_s": rw_s, "mbar_iterations": iters, "mbar": mbar,
            "phase_map": {"kT": kT_q.tolist(), "p": p_q.tolist(),
                          "N_mean": nm.reshape(12, 12).round(3).tolist(),
                          "N_most_probable": np.argmax(pN, axis=1).reshape(12, 12).tolist()}}


TWO_SPECIES = ("two LJ gases B, C over the fcc111 12x12x4 slab, 8 kT x 16 mu_B x 8 mu_C = 1024 replicas, "
               "N_B + N_C <= 256, 20 moves/sweep; step = 10 sweeps + 1 replica-exchange attempt "
               "(5 directions)")


def two_species_arm(torch, stream, flush, steps, sweeps, equil=2000, seed=0):
    """Two grand-canonical species (regc_init_grid2) at paper scale: device-
    timed steps as in the main arm, then a production run with per-state
    energy windows (convergence by the KS test of the two halves) and the
    pooled (N_B, N_C, E) histogram reweighted (Sec. II.B) onto a mu_B x mu_C
    map at three temperatures."""
    from paper_1908_11118_gb300 import Regc

    p = W.two_gas_paper_scale(seed=seed)
    rng = np.random.default_rng(seed)
    pos, n, nb = W.two_gas_initial(p, rng.integers(0, 40, p.S), rng.integers(0, 40, p.S), seed=seed)
    g = Regc(p, stream=stream)
    g.set_walkers(pos, n, nb=nb)
    g.run(equil, exchange_every=SWEEPS_PER_STEP)
    for _ in range(3):
        g.sweep(SWEEPS_PER_STEP)
        g.exchange()
    mv0, ex0, _ = g.counters()
    ev = []
    torch.cuda.synchronize()
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        g.sweep(SWEEPS_PER_STEP)
        e[1].record(stream)
        g.exchange()
        e[2].record(stream)
        ev.append(e)
    torch.cuda.synchronize()
    step_ms = sum(e[0].elapsed_time(e[2]) for e in ev) / steps
    sweep_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
    mv1, ex1, _ = g.counters()
    dm = mv1 - mv0
    dx = ex1 - ex0
    timed = {"steps": steps, "ms_per_step": step_ms, "sweep_launch_ms": sweep_ms,
             "trial_moves_per_s": p.S * SWEEPS_PER_STEP * p.moves_per_sweep / (step_ms / 1e3),
             "acceptance": float(dm[:, :, 1].sum() / max(dm[:, :, 0].sum(), 1)),
             "exchange_acceptance_per_direction": (dx[:, :, 1].sum(0) / np.maximum(dx[:, :, 0].sum(0), 1)).tolist(),
             "l2": "flushed (256 MB memset) before every timed step"}
    g.set_state_windows(1024, 0.5, None)
    g.reset_histograms()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    half, done, chunk = None, 0, 1000
    while done < sweeps:
        k = min(chunk, sweeps - done)
        g.run(k, exchange_every=SWEEPS_PER_STEP)
        done += k
        if half is None and done >= sweeps // 2:
            half = g.state_histograms()[0]
    full = g.state_histograms()[0]
    torch.cuda.synchronize()
    run_s = time.perf_counter() - t0
    ks, crit = ks_halves(half, full - half)
    h = g.histograms()
    cnt = g.species_counts()
    kT_q = np.array([p.kT[1], p.kT[len(p.kT) // 2], p.kT[-2]])
    mb = np.linspace(-6.0, -2.0, 12)
    mc = np.linspace(-6.0, -2.0, 12)
    T, MB, MC = np.meshgrid(kT_q, mb, mc, indexing="ij")
    t1 = time.perf_counter()
    nbm, ncm, pb, pc, f, iters = g.reweight2(T.ravel(), MB.ravel(), MC.ravel(), tol=1e-9, max_iter=200000)
    rw_s = time.perf_counter() - t1
    mbar = mbar_summary()
    g.close()
    shape = (len(kT_q), len(mb), len(mc))
    return {"workload": TWO_SPECIES, "equilibration_sweeps": equil, "timed": timed,
            "production": {"sweeps": sweeps, "run_s": run_s,
                           "trial_moves_per_s": p.S * sweeps * p.moves_per_sweep / run_s,
                           "observations": int(h["omega"].sum()),
                           "pooled_bins_occupied": int(np.count_nonzero(h["hNE"])),
                           "e_out": int(h["e_out"].sum()),
                           "walkers_N_B_mean": float(cnt.mean()),
                           "convergence_ks_halves": {"median": float(np.median(ks)), "max": float(np.max(ks)),
                                                     "states_unchanged_at_1pct": int(np.sum(ks < crit))}},
            "reweight_s": rw_s, "mbar_iterations": iters, "mbar": mbar,
            "phase_map": {"kT": kT_q.tolist(), "mu_B": mb.tolist(), "mu_C": mc.tolist(),
                          "N_B_mean": nbm.reshape(shape).round(2).tolist(),
                          "N_C_mean": ncm.reshape(shape).round(2).tolist(),
                          "N_B_most_probable": np.argmax(pb, axis=1).reshape(shape).tolist(),
                          "N_C_most_probable": np.argmax(pc, axis=1).reshape(shape).tolist()}}


def mbar_summary():
    """The last MBAR solve (regc_mbar_last_info) with the sparse maps' rate:
    algorithmic bytes per map = 24 per kept entry (index + FP64 value, by bin
    and by state) + 32 per bin (row pointer, H_b, V_b written and read)."""
    from paper_1908_11118_gb300 import mbar_last_info
    i = mbar_last_info()
    per_map = 24.0 * i["nnz"] + 32.0 * i["B"]
    gbs = per_map * i["sparse_maps"] / (i["ms_maps"] / 1e3) / 1e9 if i["ms_maps"] > 0 else None
    peak, src = hbm_peak()
    return dict(i, bytes_per_map=per_map, sparse_map_gbs=gbs,
                sparse_map_frac_of_hbm=(gbs / peak if gbs else None), hbm_peak_source=src,
                kept_fraction=i["nnz"] / max(1, i["S"] * i["B"]))


def paper_structure_spec(p):
    """Slabs of 0.12 A over the 48 A zone (Sec. III.A) and three adsorbate
    layers above the floor for g_xy, lateral bins of 0.1 A up to 4.9 A (the
    inscribed radius of the hexagonal cell is 4.97 A)."""
    return {"n_z": 400, "dz": 0.12,
            "layers": [(p.z_lo, p.z_lo + 0.6), (p.z_lo + 0.6, p.z_lo + 1.6), (p.z_lo + 1.6, p.z_lo + 2.6)],
            "n_r": 49, "dr": 0.1}


def rho_u_convergence(p, smp):
    """The paper's convergence criterion (Sec. III.A: the density of
    reduced-energy states rho(U), U = beta (E - mu N), no longer changes with
    more steps) as a diagnostic: per state, the two-sample Kolmogorov-Smirnov
    distance between the U samples of the first and second half of the
    samples held, against its 1 % critical value 1.63 sqrt(2 / n)."""
    st, N, E = smp["state"], smp["N"].astype(np.float64), smp["E"]
    beta = 1.0 / np.asarray(p.kT)[st // p.M]
    U = beta * (E - np.asarray(p.mu)[st % p.M] * N)
    half = len(st) // 2
    ks, ok = [], 0
    for s in range(p.S):
        a = np.sort(U[:half][st[:half] == s])
        b = np.sort(U[half:][st[half:] == s])
        if len(a) < 5 or len(b) < 5:
            continue
        grid = np.concatenate([a, b])
        d = np.max(np.abs(np.searchsorted(a, grid, side="right") / len(a) -
                          np.searchsorted(b, grid, side="right") / len(b)))
        ks.append(d)
        ok += d < 1.63 * np.sqrt((len(a) + len(b)) / (len(a) * len(b)))
    ks = np.array(ks)
    return {"states": int(len(ks)), "ks_median": float(np.median(ks)) if len(ks) else None,
            "ks_max": float(np.max(ks)) if len(ks) else None,
            "states_unchanged_at_1pct": int(ok),
            "note": "samples are correlated (one per 100 steps), so the critical value is optimistic"}


def paper_cycle_arm(torch, stream, flush, n_steps, chunk=1000, x0=0.99, n_c=10, cpu_seconds=8.0, seed=0,
                    sample_every=100):
    """The paper's whole LJ sampling run through regc_cycle: n_steps REGC steps
    of the 160 replicas from the pristine slab (N_B = 0 everywhere), with the
    structure of every replica sampled every `sample_every` steps as the paper
    sub-samples; device-timed in chunks of `chunk` steps with the L2 flushed
    before each.  Reports the rate, the wall time of the run, the
    replica-exchange acceptance (about 25 % in the paper), the mean and modal
    N_B per state from the second half counted per A18 cell, and the MBAR
    reweighting of the samples per phase (Eq. avegr) with the HBM roofline of
    its accumulation kernel."""
    from paper_1908_11118_gb300 import Regc
    p = W.lj_a18_hex_slab(seed=seed)
    spec = paper_structure_spec(p)
    g = Regc(p, stream=stream)
    g.set_walkers(np.zeros((p.S, p.nmax, 3)), np.zeros(p.S, np.int32))
    g.structure_init(spec["n_z"], spec["dz"], spec["layers"], spec["n_r"], spec["dr"],
                     (n_steps // sample_every + 1) * p.S)
    g.cycle(200, x0, n_c)                       # warm-up: launches and first insertions
    g.reset_histograms()
    mv0, ex0, _ = g.counters()
    ev, n_ex = [], 0
    h_half = None
    done = 0
    torch.cuda.synchronize()
    while done < n_steps:
        k = min(chunk, n_steps - done)
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        left = k
        while left > 0:
            step = min(sample_every, left)
            n_ex += g.cycle(step, x0, n_c)
            left -= step
            if step == sample_every:
                g.structure_sample()
        b.record(stream)
        ev.append((a, b))
        done += k
        if h_half is None and done >= n_steps // 2:
            h_half = g.histograms()["hN"]
            g.structure_reset()                 # MBAR on the second half only
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    mv1, ex1, _ = g.counters()
    h = g.histograms()["hN"] - h_half
    ex = (ex1 - ex0).sum(axis=(0, 1))
    trials = int((mv1[:, :, 0] - mv0[:, :, 0]).sum())
    nv = np.arange(p.nmax + 1)
    mean_nb = (h @ nv) / np.maximum(h.sum(axis=1), 1)
    mode_nb = np.argmax(h, axis=1)
    modes, counts = np.unique(mode_nb, return_counts=True)
    drift = g.check_energy()
    wpw = g.warps_per_walker()

    # MBAR over the sub-sampled second half, per phase, at eight states: the
    # sampled corners and the two state points of the paper's g_xy figure
    n_samples = g.structure_count()
    conv = rho_u_convergence(p, g.structure_get())
    kB = W.K_B_EV
    # the corner states, a few inside the grid, and the paper's two g_xy state
    # points given as (T, p): (200 K, 2.03e-17 atm) and (600 K, 8.89e-2 atm)
    from paper_1908_11118_gb300 import mu_of_pressure
    kq = np.array([kB * 200, kB * 650, kB * 200, kB * 650, kB * 425, kB * 300, kB * 200, kB * 600])
    mq = np.concatenate([[-0.9, -0.9, -2.4, -2.4, -1.5, -1.9],
                         mu_of_pressure(kq[6:], np.array([2.03e-17, 8.89e-2]) * W.ATM_EV_PER_A3, p.lambda0)])
    t0 = time.perf_counter()
    rw = g.structure_reweight(kq, mq, 0, p.nmax, tol=1e-9, max_iter=200000)
    rw_s = time.perf_counter() - t0
    tm = g.structure_timing()
    # MBAR@REGC against aiAT@REGC (Sec. III.A.1) on a (T, mu) grid: the most
    # probable N_B against the composition of lowest formation free energy
    Tg, mg = np.meshgrid(200.0 + 50.0 * np.arange(10), -2.4 + 0.05 * np.arange(31), indexing="ij")
    rg = g.structure_reweight(kB * Tg.ravel(), mg.ravel(), 0, p.nmax, tol=1e-9, max_iter=200000)
    mbar_phase = np.argmax(rg["p"], axis=1)
    _, _, ai_phase = g.aiat(mg.ravel())
    low = ai_phase <= 18                      # up to the first monolayer of the A18 cell
    agree = {"all": float(np.mean(mbar_phase == ai_phase)),
             "aiat_nb_le_18": float(np.mean((mbar_phase == ai_phase)[low])) if low.any() else None,
             "aiat_nb_gt_18": float(np.mean((mbar_phase == ai_phase)[~low])) if (~low).any() else None,
             "mbar_minus_aiat_nb_mean": float(np.mean(mbar_phase - ai_phase)),
             "grid": "10 T (200-650 K) x 31 mu (-2.4..-0.9 eV, 0.05 eV)"}
    ach = tm["bytes_accumulate"] / (tm["ms_accumulate"] / 1e3) / 1e9
    peak, peak_src = hbm_peak()
    phases = []
    for q in range(len(kq)):
        i = int(np.argmax(rw["p"][q]))
        phases.append({"T_K": round(kq[q] / kB), "mu_eV": round(float(mq[q]), 4), "most_probable_nb": i,
                       "p": round(float(rw["p"][q, i]), 3), "p_nb_59": float(rw["p"][q, 59])})
    g.close()
    # the oracle on the same run for a bounded number of steps, on the host cores
    from oracle import oracle as O
    O.build()
    o = O.Oracle(p)
    o.cycle(200, x0, n_c, hist=False)
    chunks_cpu, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < cpu_seconds and chunks_cpu < len(ev):
        o.cycle(chunk, x0, n_c, hist=True)
        chunks_cpu += 1
    el = time.perf_counter() - t0
    steps_cpu = chunks_cpu * chunk
    # the GPU on the same leading chunks of the same run (both from the
    # pristine slab, same seed), for a like-for-like ratio
    ms_same = sum(a.elapsed_time(b) for a, b in ev[:chunks_cpu])
    return {
        "workload": PAPER_CYCLE,
        "steps": n_steps,
        "ms": ms,
        "regc_steps_per_s": n_steps / (ms / 1e3),
        "trial_moves_per_s": trials / (ms / 1e3),
        "paper_run_seconds": 1.2e5 * ms / 1e3 / n_steps,
        "warps_per_walker": wpw,
        "replica_exchange_steps": n_ex,
        "replica_exchange_acceptance": float(ex[1] / max(ex[0], 1)),
        "mean_nb": np.round(mean_nb.reshape(p.L, p.M), 1).tolist(),
        "modal_nb": {str(int(m)): int(c) for m, c in zip(modes, counts)},
        "energy_drift": drift,
        "l2": "flushed (256 MB memset) before every chunk of %d steps" % chunk,
        "structure": {
            "samples": n_samples, "every_steps": sample_every, "spec": {k: v for k, v in spec.items()},
            "reweight_s": rw_s, "mbar_iterations": rw["iters"], "ms_mbar": tm["ms_mbar"],
            "ms_weights": tm["ms_weights"], "ms_accumulate": tm["ms_accumulate"],
            "most_probable_phase": phases,
            "mbar_vs_aiat": agree,
            "rho_u_convergence": conv,
            "roofline": {"bound": "hbm", "kernel": "accumulate_kernel", "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak, "traffic": None, "peak_source": peak_src,
                         "work": "%.4g algorithmic bytes per launch (%d samples x %d query states)"
                                 % (tm["bytes_accumulate"], n_samples, len(kq))},
        },
        "cpu_baseline": {"value": steps_cpu / el, "unit": "REGC steps/s", "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": "the first %d steps of the same run from the pristine slab, after the "
                                   "same 200 warm-up steps, without structure samples (%.1f s)" % (steps_cpu, el),
                         "gpu_same_steps_per_s": steps_cpu / max(ms_same / 1e3, 1e-9)},
    }


# ---------------------------------------------------------------- own arm

def run_own(args):
    import torch

    from paper_1908_11118_gb300 import Regc
    from paper_1908_11118_gb300 import build as B

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = W.fcc111_paper_scale(seed=rank)
    pos0, n0 = initial_state(p, rank)
    stream = torch.cuda.Stream()
    g = Regc(p, stream=stream)
    g.set_walkers(pos0, n0)
    g.run(args.equil, exchange_every=SWEEPS_PER_STEP)
    for _ in range(args.warmup):
        g.sweep(SWEEPS_PER_STEP)
        g.exchange()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    mv0, _, pr0 = g.counters()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for k in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        g.sweep(SWEEPS_PER_STEP)
        ev[k][1].record(stream)
        g.exchange()
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(K)]
    sweep_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    mv1, _, pr1 = g.counters()
    total_ms = float(sum(step_ms))
    moves = p.S * SWEEPS_PER_STEP * p.moves_per_sweep * K
    value, total_max = job_throughput(total_ms, moves, world, "cuda")
    accepted = int((mv1[:, :, 1] - mv0[:, :, 1]).sum())
    pairs = int(pr1[0] - pr0[0])
    cand = int(pr1[1] - pr0[1])
    rounds = int(pr1[2] - pr0[2])
    evals = int(pr1[3] - pr0[3])
    mean_sweep_s = sum(sweep_ms) / K / 1e3
    achieved = pairs / K * FLOPS_PER_PAIR / mean_sweep_s / 1e12
    peak, peak_src = fp32_peak(stream)

    # end to end through the C ABI with pinned host buffers: full walker state
    # in (set_walkers: positions, N, labels; energies recomputed on the device),
    # one step, full walker state and energies out, every step
    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()
    host = (pinned((p.S, p.nmax, 3), torch.float32), pinned((p.S,), torch.int32),
            pinned((p.S,), torch.float64), pinned((p.S,), torch.int32))
    g.get_walkers(out=host)
    pos_h, n_h, e_h, sow_h = host
    e2e_steps = max(1, args.e2e_steps)
    for _ in range(2):   # warm-up of the host path, whole steps
        g.set_walkers(pos_h, n_h, sow_h)
        g.sweep(SWEEPS_PER_STEP)
        g.exchange()
        g.get_walkers(out=host)
    torch.cuda.synchronize()
    # the harness's own garbage collection stays out of the timed loop
    gc_was_enabled = gc.isenabled()
    gc.disable()
    e2e_each = []
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ts = time.perf_counter()
        g.set_walkers(pos_h, n_h, sow_h)
        g.sweep(SWEEPS_PER_STEP)
        g.exchange()
        g.get_walkers(out=host)
        e2e_each.append(time.perf_counter() - ts)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if gc_was_enabled:
        gc.enable()
    h2d = p.S * p.nmax * 12 + p.S * 4 * 2
    d2h = p.S * p.nmax * 12 + p.S * (4 + 8 + 4) + 4

    regcmd = None
    if args.md and rank == 0:
        regcmd = regcmd_arm(g, p, torch, stream, flush, args.md_segments)

    batched = None
    if args.batch and rank == 0:
        batched = batched_uneven_arm(torch, args.batch_steps)

    da = None
    if args.da and rank == 0:
        da = [delayed_acceptance_arm(W.fcc100_small(seed=0), DA_SMALL, torch, stream, flush, 1_000_000,
                                     args.da_train_steps, args.da_steps_small),
              delayed_acceptance_arm(p, WORKLOAD, torch, stream, flush, 1_000_000, args.da_train_steps,
                                     args.da_steps_large)]
    cluster = None
    if args.cluster and rank == 0:
        # the cluster-in-gas workload: plain and delayed acceptance, same protocol
        cluster = delayed_acceptance_arm(W.cluster_in_gas(seed=0), CLUSTER_WORKLOAD, torch, stream, flush,
                                         1_000_000, args.da_train_steps, args.da_steps_large)

    paper = None
    if args.paper_cycle and rank == 0:
        paper = paper_cycle_arm(torch, stream, flush, args.paper_steps)

    production = None
    if args.production > 0 and rank == 0:
        production = production_arm(torch, stream, args.production)

    cluster_prod = None
    if args.cluster_production > 0 and rank == 0:
        cluster_prod = cluster_production_arm(torch, stream, args.cluster_production, 1_000_000,
                                              args.da_train_steps)

    two = None
    if args.two_species and rank == 0:
        two = two_species_arm(torch, stream, flush, args.two_species_steps, args.two_species_sweeps)

    line = None
    if rank == 0:
        cpu = None
        if world == 1:
            rate, steps, el, cores, orc = time_oracle(p, pos0, n0, seconds=args.cpu_seconds, equil=args.equil)
            rate1, steps1, el1, _, _ = time_oracle(p, pos0, n0, seconds=args.cpu_seconds / 4, threads=1, orc=orc)
            cpu = {"value": rate, "unit": "moves/s", "cores": cores, "kind": "oracle",
                   "sample": "full 1024-replica workload from the seeded lattice state after %d "
                             "equilibration sweeps of the oracle's own, %d steps of 10 sweeps + "
                             "exchange (%.1f s)" % (args.equil, steps, el),
                   "value_1_thread": rate1,
                   "sample_1_thread": "%d steps on one thread (%.1f s)" % (steps1, el1)}
        line = {
            "metric": METRIC, "value": value, "unit": "moves/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(args),
            "precision": "pair energies f32, totals exact 64-bit fixed point, acceptance f64",
            "accepted_moves_per_s": accepted * world / (total_max / 1e3),
            "pair_interactions_per_s": pairs * world / (total_max / 1e3),
            "candidate_pairs_per_s": cand * world / (total_max / 1e3),
            "roofline": {"bound": "alu", "kernel": "sweep_kernel", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": SWEEP_TRAFFIC_BYTES,
                         "peak_source": peak_src,
                         "work": "%d flop/pair x pairs within rc (%.3g per launch)" % (FLOPS_PER_PAIR, pairs / K),
                         "launch_ms": mean_sweep_s * 1e3},
            "e2e": {"value": p.S * SWEEPS_PER_STEP * p.moves_per_sweep * world / e2e_s, "unit": "moves/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "ms_per_step_mean": e2e_s * 1e3,
                    "ms_per_step_median": statistics.median(e2e_each) * 1e3, "ms_per_step_max": max(e2e_each) * 1e3},
            "speculation": {"warps_per_walker": g.warps_per_walker(),
                            "moves_per_round": moves / max(rounds, 1),
                            "kept_fraction": moves / max(evals, 1)},
            "gpu_launches": 2 * K,
            "clocks": clk,
            "cpu_baseline": cpu,
            "surrogate_da": da,
            "batched_uneven": batched,
            "regcmd": regcmd,
            "cluster_in_gas": cluster,
            "paper_lj_cycle": paper,
            "production_phase_map": production,
            "two_species": two,
            "cluster_production": cluster_prod,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_own(args)


if __name__ == "__main__":
    sys.exit(main())
