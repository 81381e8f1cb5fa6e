"""Benchmark: walker-steps per second of the GFK helium walk on one GB300.

One bench step = one full run of a workload through the C ABI; the default
(the headline) is:
initialise 2^20 walkers of the He 1^1S trial function
exp(-2 r1 - 2 r2) exp(r12 / (2 (1 + 0.5 r12))) and advance them 20000 moves at
dt = 0.005 on the mixed-precision path (FP32 drift / local energy / normals,
FP64 log-weights and population sums), with the population sums of every move.
The same line carries the FP64 path on the same seeds (speed and the mixed
path's energy error), the rooflines of the walk kernel (FP32 flops counted on
the oracle's procedure against the measured FFMA rate; special-function unit;
issue slots), and, under "workloads", the 2^3S, twelve-instance batched and
+-1 Bernoulli walks and the adjoint gradient with 50 Adam steps, each measured
on its own.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
population (its own Philox stream) -- weak scaling, no collective on the data
path; the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/sec on 1 GB300 (FP32-mixed vs FP64) at stated energy error vs FP64 oracle"
UNIT = "walker-steps/s"
WORKLOADS = {
    "ground": ("He 1^1S ground state: 2^20 walkers x 20000 moves, dt=0.005, trial "
               "exp(-2r1-2r2)exp(r12/(2(1+0.5r12))), E_T=-2.9037, Philox seed 0, mixed FP32 "
               "physics / FP64 weights"),
    "triplet": ("He 2^3S: 2^20 walkers x 20000 moves, dt=0.0025, trial "
                "(e^{-2r1-0.5r2}-e^{-0.5r1-2r2})exp(r12/(4(1+0.3r12))), node r1=r2 by kill, "
                "E_T=-2.1752, mixed"),
    "adjoint": ("gradient of the final space-averaged 1^1S energy w.r.t. [Z, a, beta, c1..c4]: "
                "2^18 walkers x 2000 moves, dt=0.005, checkpoints every 64 moves, FP32 forward "
                "with FP64 weights (gfk_grad: forward + recompute + reverse sweep)"),
    "bernoulli": ("He 1^1S with the paper's own +-1 walk: 2^20 walkers x 20000 moves, "
                  "dt=1/900 (scale 30, step length 1/30), Superduper generators "
                  "S=(69069 S+1) mod 2^32 per walker, same trial and E_T as ground, mixed"),
    "batched": ("12 instances {1^1S, 2^3S, P_z} x dt {0.01,0.005,0.0025,0.00125}, walker counts "
                "round(2^U), U~U[16,21] (numpy default_rng(1)), sum 7.75e6 walkers x 10000 moves, "
                "one launch per chunk, mixed"),
}
SEED = 0

# Algorithmic work of one walker-step, counted on the oracle's own procedure by
# oracle/opcount.py (tests/test_op_counts.py checks that these literals equal its
# output): "flops" = floating-point additions, multiplications and divisions (a
# fused multiply-add is two), "special" = square roots, exponentials,
# logarithms, sines and cosines, "int" = the integer operations of the noise.
# Keyed by (noise, trial case); the cases are the workloads' trial functions
# per state (0: the 1^1S product, 1: the 2^3S pair, 2: the P_z pair).
OP_COUNTS = {
    (0, "ground"): {"flops": 168.0, "special": 18.0, "int": 68.0, "fp_add": 56.0,
                    "fp_mul": 87.0, "fp_div": 25.0, "fp_sqrt": 6.0, "fp_exp": 3.0,
                    "fp_log": 3.0, "fp_sin": 3.0, "fp_cos": 3.0},
    (0, "triplet_2s3"): {"flops": 212.0, "special": 20.0, "int": 68.0, "fp_add": 67.0,
                         "fp_mul": 112.0, "fp_div": 33.0, "fp_sqrt": 6.0, "fp_exp": 5.0,
                         "fp_log": 3.0, "fp_sin": 3.0, "fp_cos": 3.0},
    (0, "pz"): {"flops": 224.0, "special": 20.0, "int": 68.0, "fp_add": 71.0, "fp_mul": 118.0,
                "fp_div": 35.0, "fp_sqrt": 6.0, "fp_exp": 5.0, "fp_log": 3.0, "fp_sin": 3.0,
                "fp_cos": 3.0},
    (1, "ground"): {"flops": 138.0, "special": 6.0, "int": 12.0, "fp_add": 50.0,
                    "fp_mul": 63.0, "fp_div": 25.0, "fp_sqrt": 3.0, "fp_exp": 3.0,
                    "fp_log": 0.0, "fp_sin": 0.0, "fp_cos": 0.0},
    (1, "triplet_2s3"): {"flops": 182.0, "special": 8.0, "int": 12.0, "fp_add": 61.0,
                         "fp_mul": 88.0, "fp_div": 33.0, "fp_sqrt": 3.0, "fp_exp": 5.0,
                         "fp_log": 0.0, "fp_sin": 0.0, "fp_cos": 0.0},
    (1, "pz"): {"flops": 194.0, "special": 8.0, "int": 12.0, "fp_add": 65.0, "fp_mul": 94.0,
                "fp_div": 35.0, "fp_sqrt": 3.0, "fp_exp": 5.0, "fp_log": 0.0, "fp_sin": 0.0,
                "fp_cos": 0.0},
}
STATE_CASE = {0: "ground", 1: "triplet_2s3", 2: "pz"}
# Each special operation of the count runs as one special-function-unit
# instruction on the GPU; the measured rate of that instruction class
# (gfk_measure_peak) prices it: square root -> rsqrt, exponential -> ex2,
# logarithm -> lg2, sine and cosine -> sin.
SPECIAL_UNIT = {"fp_sqrt": "rsq", "fp_exp": "ex2", "fp_log": "lg2", "fp_sin": "sin",
                "fp_cos": "sin"}
# Issue slots: 4 schedulers x 32 lanes per SM and clock.
LANES_PER_SM_CLK = 128
# ncu figures of the mixed walk kernels at the bench's launch shape (2^20 walkers x
# 1024 moves, 128 threads x 2 walkers; one capture per (state, noise) kernel:
# `bench.py --profile-case --profile-walkers 1048576 --profile-moves 1024
# --profile-state S --noise N`), valid only for the kernel sources they were taken
# on (sha256 prefix of WALK_SOURCES' code, comments and layout aside: _src_sha):
# DRAM bytes (read + write) and executed thread
# instructions per walker-step, the issue-active fraction and the busiest pipe (the
# FMA-heavy pipe, which also runs the integer multiplies of the Philox rounds).
WALK_PROFILE = {       # (state, noise) -> capture of that walk kernel
    (0, 0): {"src_sha": "8c28c12f7806baf6", "bytes_per_walker_step": 0.19932,
             "inst_per_walker_step": 189.1, "issue_active": 0.695, "fmaheavy_active": 0.694},
    (0, 1): {"src_sha": "8c28c12f7806baf6", "bytes_per_walker_step": 0.19865,
             "inst_per_walker_step": 132.2, "issue_active": 0.696, "fmaheavy_active": 0.656},
    (1, 0): {"src_sha": "8c28c12f7806baf6", "bytes_per_walker_step": 0.19963,
             "inst_per_walker_step": 227.2, "issue_active": 0.695, "fmaheavy_active": 0.690},
    (2, 0): {"src_sha": "8c28c12f7806baf6", "bytes_per_walker_step": 0.19973,
             "inst_per_walker_step": 252.5, "issue_active": 0.681, "fmaheavy_active": 0.717},
}




# Sources the mixed walk kernel is compiled from (the kernels and the device
# code they include); a captured figure holds only while their code is
# unchanged (comments and layout aside).
WALK_SOURCES = tuple("paper_1703_08977_gb300/csrc/" + f for f in (
    "gfk_mixed.cuh", "gfk_mixed.cu", "gfk_mixed_bern.cu", "gfk_device.cuh", "gfk_block.cuh",
    "gfk_types.h", "gfk_lanes.cuh", "gfk_eval_f32.cuh", "gfk_debug.h"))


def _code_tokens(text: str) -> str:
    """C++ source without its comments, each run of whitespace one space (string and
    character literals, such as inline PTX, kept as written)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def _src_sha() -> str:
    h = hashlib.sha256()
    for f in WALK_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(_code_tokens(fh.read()).encode())
    return h.hexdigest()[:16]


def _op_counts(insts):
    """Walker-count-weighted op counts per walker-step of a workload's instances."""
    n = sum(d["n_walkers"] for d in insts)
    out = {}
    for d in insts:
        c = OP_COUNTS[(d["noise"], STATE_CASE[d["state"]])]
        for k, v in c.items():
            out[k] = out.get(k, 0.0) + v * d["n_walkers"] / n
    return out


def bench_config(name, rank=0):
    """The `config` object of a workload (the same for both arms of the bench)."""
    insts, moves = _workload(name, rank)
    n = sum(d["n_walkers"] for d in insts)
    return {"workload": WORKLOADS[name], "name": name, "walkers_per_gpu": n, "moves": moves,
            "l2": f"flushed (256 MB write) before every timed step; state {n * 33 / 2**20:.0f} MB"}


# ----------------------------------------------------------------------------
def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # scratch file of the samples (the JSON line carries their summary);
        # GFK_CLOCKS_DIR keeps it somewhere else than the system temp folder
        self.path = os.path.join(os.environ.get("GFK_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"gfk_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
def run_reference(args):
    """The oracle (plain FP64 C, unchanged) on a bounded sample of the workload, on all
    host cores: one spawned process per core walks a disjoint block of walker ids."""
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    name = args.workload if args.workload in ("ground", "bernoulli") else "ground"
    n_sample, moves = 1 << 14, 100
    with OraclePool() as pool:
        for _ in range(args.warmup):
            pool.walk(name, n_sample, moves)
        t = [pool.walk(name, n_sample, moves) for _ in range(args.steps)]
        cores = pool.n
    dt_s = sum(t)
    value = n_sample * moves * args.steps / dt_s
    sample = (f"{n_sample} walkers x {moves} moves per step (a slice of the workload), "
              f"{cores} processes over disjoint walker ids")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(name),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _oracle_block(job):
    """One process's share of an oracle timing: walker ids [lo, hi) for `moves` moves;
    returns the seconds it took (module level, so spawned processes can run it)."""
    name, lo, hi, moves = job
    import numpy as np
    import oracle
    kind, params, dt, et, noise = _oracle_case(name)
    t0 = time.perf_counter()
    w = oracle.Walk(kind, params, ids=np.arange(lo, hi, dtype=np.uint32), dt=dt, e_trial=et,
                    seed=SEED, noise=noise)
    w.advance(moves)
    return time.perf_counter() - t0


class OraclePool:
    """Spawned worker processes (spawn: the parent may already hold a CUDA context)."""

    def __init__(self, n=None):
        # one process per host core, at most 64 (start-up cost on very large hosts)
        self.n = n or max(1, min(64, os.cpu_count() or 1))

    def __enter__(self):
        import multiprocessing as mp
        self.pool = mp.get_context("spawn").Pool(self.n)
        # each worker imports the oracle once before anything is timed
        self.pool.map(_oracle_block, [("ground", 0, 1, 1)] * self.n)
        return self

    def __exit__(self, *exc):
        self.pool.close()
        self.pool.join()

    def walk(self, name, n_walkers, moves):
        """Wall-clock seconds for n_walkers x moves, split into one block per process."""
        edges = [n_walkers * i // self.n for i in range(self.n + 1)]
        jobs = [(name, edges[i], edges[i + 1], moves) for i in range(self.n)
                if edges[i + 1] > edges[i]]
        t0 = time.perf_counter()
        self.pool.map(_oracle_block, jobs, chunksize=1)
        return time.perf_counter() - t0


def _oracle_case(name):
    """(kind, params, dt, E_T, noise) of the ground-state workloads for the oracle."""
    if name == "bernoulli":
        return 0, [2.0, 0.5, 0.5], 1.0 / 900.0, -2.9037, 1
    return 0, [2.0, 0.5, 0.5], 0.005, -2.9037, 0


def cpu_baseline(name="ground"):
    """The oracle on the host: all cores (one spawned process per core, disjoint walker
    ids; the reported value) and one thread (reported beside it)."""
    import oracle
    oracle.build()
    moves = 600
    t1 = _oracle_block((name, 0, 1 << 13, moves))
    single = (1 << 13) * moves / t1
    with OraclePool() as pool:
        n_par = (1 << 13) * pool.n
        tp = pool.walk(name, n_par, moves)
        cores = pool.n
    return {"value": n_par * moves / tp, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_par} walkers x {moves} moves of the same workload, {cores} processes "
                      "over disjoint walker ids (2^13 each)",
            "single_thread": {"value": single, "sample": f"2^13 walkers x {moves} moves"}}


def _workload(name, rank):
    from paper_1703_08977_gb300 import workloads as wl
    if name == "ground":
        insts, moves = wl.ground_at_scale(0.005)
    elif name == "triplet":
        insts, moves = wl.triplet_at_scale()
    elif name == "bernoulli":
        insts, moves = wl.bernoulli_at_scale()
    else:
        insts, moves = wl.batched()
    for d in insts:
        # each rank advances its own walker ids of one global population
        # (weak scaling: the population grows with the number of ranks)
        d["walker_id0"] = rank * d["n_walkers"]
    return insts, moves


def measure_peaks():
    """Measured lane-operation rates (per second, whole GPU) of the instruction classes
    the rooflines use: FP32 and FP64 fused multiply-add and the special-function unit's
    ex2, rsqrt, lg2 and sin (gfk_measure_peak, about 10 ms each)."""
    from paper_1703_08977_gb300 import gfk
    return {op: gfk.gfk_measure_peak(op)
            for op in ("ffma", "ffma2", "dfma", "ex2", "rsq", "lg2", "sin")}


def _walk_profile(insts):
    """The ncu figures of a workload's walk kernels, averaged over its instances by
    walker count (one kernel per (state, noise) pair); None if a kernel has no capture
    of the current sources."""
    sha = _src_sha()
    keys = ("bytes_per_walker_step", "inst_per_walker_step", "issue_active", "fmaheavy_active")
    acc = dict.fromkeys(keys, 0.0)
    total = 0
    for d in insts:
        p = WALK_PROFILE.get((d["state"], d["noise"]))
        if p is None or p["src_sha"] != sha:
            return None
        for k in keys:
            acc[k] += p[k] * d["n_walkers"]
        total += d["n_walkers"]
    return {k: v / total for k, v in acc.items()}


def walk_rooflines(name, insts, avg_launch_ms, ws_per_launch, peaks, n_sm, sm_max, sm_mhz):
    """The walk kernel's rooflines from its own launch time: FP32 flops against the
    measured FFMA rate (the primary figure), the special-function unit against its
    measured rates, and issue slots from the ncu instruction count."""
    counts = _op_counts(insts)
    rate = ws_per_launch / (avg_launch_ms / 1e3)          # walker-steps/s in the walk kernel
    achieved = counts["flops"] * rate / 1e12
    # the FP32 multiply-add rate, scalar or packed, whichever is higher
    fma_rate = max(peaks["ffma"], peaks.get("ffma2", 0.0))
    peak = 2.0 * fma_rate / 1e12
    derived = n_sm * LANES_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
    prof = _walk_profile(insts)
    valid = prof is not None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": prof["bytes_per_walker_step"] * ws_per_launch if valid else None,
            "kernel": "walk_mixed_kernel",
            "peak_basis": "of measured: the higher of the FFMA and packed FFMA2 lane rates "
                          "(gfk_measure_peak, this run) x 2 flops",
            "peak_derived": derived, "frac_of_derived": achieved / derived,
            "derived_basis": f"{n_sm} SMs x {LANES_PER_SM_CLK} FP32 lanes x 2 flops x "
                             f"{sm_max:.0f} MHz",
            "flops_per_walker_step": counts["flops"],
            "counts": "oracle/opcount.py (the oracle's walker-step on a counting scalar)",
            "avg_launch_ms": avg_launch_ms, "walker_steps_per_launch": ws_per_launch}
    busy = sum(counts[k] / peaks[u] for k, u in SPECIAL_UNIT.items())   # s per walker-step
    mufu = {"frac": busy * rate, "special_per_walker_step": counts["special"],
            "basis": "sum over sqrt, exp, log, sin, cos of count / measured rate of "
                     "rsq, ex2, lg2, sin"}
    clk = (sm_mhz or sm_max) * 1e6
    inst = prof.get("inst_per_walker_step") if valid else None
    issue = {"frac": inst * rate / (n_sm * LANES_PER_SM_CLK * clk) if inst else None,
             "inst_per_walker_step": inst, "ncu_issue_active": prof.get("issue_active") if valid else None,
             "ncu_fmaheavy_pipe_active": prof.get("fmaheavy_active") if valid else None,
             "basis": f"executed thread instructions (ncu) / ({n_sm} SMs x {LANES_PER_SM_CLK} "
                      "issue lanes x sampled SM clock)"}
    return roof, mufu, issue


def measure_adjoint(steps, warmup, adam=True):
    """Workload 5: walker-steps/s of gfk_grad (each walker-step counted once although it is
    walked forward, recomputed and swept backwards), mixed and FP64, the mixed
    gradient's error against the FP64 one, and the 50-step Adam variance minimisation."""
    import numpy as np
    import torch
    from paper_1703_08977_gb300 import gfk, tuning
    n, S, K, dt = 1 << 18, 2000, 64, 0.005
    theta = [2.0, 0.5, 0.5, 0.0, 0.0, 0.0, 0.0]
    res = {}
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    for prec, name in ((gfk.GFK_PREC_MIXED, "mixed"), (gfk.GFK_PREC_FP64, "fp64")):
        d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=-2.9037, seed=SEED, prec=prec)
        with gfk.Context([d], trials=[(0, theta)]) as ctx:
            reps = steps if prec == gfk.GFK_PREC_MIXED else 1
            for _ in range(warmup if prec == gfk.GFK_PREC_MIXED else 1):
                gfk.gfk_grad(ctx.handle, 0, 0, S, K)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                loss, g = gfk.gfk_grad(ctx.handle, 0, 0, S, K)
            el = (time.perf_counter() - t0) / reps
            res[name] = {"value": n * S / el, "seconds": el, "loss": loss, "grad": g.tolist()}
            if prec == gfk.GFK_PREC_MIXED:
                # the whole trajectory kept in HBM (ckpt_every 0): no recompute
                gfk.gfk_grad(ctx.handle, 0, 0, S, 0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(reps):
                    loss0, g0 = gfk.gfk_grad(ctx.handle, 0, 0, S, 0)
                el0 = (time.perf_counter() - t0) / reps
                res["stored"] = {"value": n * S / el0, "seconds": el0,
                                 "bitwise_equal": bool(np.array_equal(g0, g) and loss0 == loss)}
    clk = clocks.stop()
    gerr = np.abs(np.array(res["mixed"]["grad"]) - np.array(res["fp64"]["grad"])).max() / \
        np.abs(np.array(res["fp64"]["grad"])).max()
    out = {"metric": "gradient walker-steps/sec on 1 GB300 (adjoint through the walk)",
           "value": res["mixed"]["value"], "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": 1e3 * res["mixed"]["seconds"], "dtype": "f32+f64",
           "config": {"workload": WORKLOADS["adjoint"], "name": "adjoint"},
           "fp64_path": {"value": res["fp64"]["value"], "unit": UNIT,
                         "mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"]},
           "gradient_mixed_vs_fp64_rel": float(gerr),
           "gradient_mixed": res["mixed"]["grad"], "gradient_fp64": res["fp64"]["grad"],
           "stored_trajectory": {
               "value": res["stored"]["value"], "unit": UNIT,
               "ms_per_step": 1e3 * res["stored"]["seconds"],
               "trajectory_bytes": 24 * n * (S + 1),
               "gradient_bitwise_equal_to_checkpointed": res["stored"]["bitwise_equal"],
               "note": "ckpt_every 0: the forward keeps every position in HBM and the reverse "
                       "sweep reads them instead of recomputing 64-move segments"},
           "gpu_launches": 5 + 2 * ((S + K - 1) // K) + 1,
           "clocks": {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
           "roofline": None,
           "roofline_note": "the reverse sweep has no algorithmic op count (the counter covers "
                            "the forward walker-step); ncu figures of its kernel are under "
                            "profiles/"}
    if adam:
        d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=-2.9037, seed=SEED,
                             prec=gfk.GFK_PREC_MIXED)
        with gfk.Context([d], trials=[(0, theta)]) as ctx:
            t0 = time.perf_counter()
            hist, th = tuning.tune(ctx.handle, 0, theta, steps=50, lr=1e-2, loss_kind=1,
                                   n_steps=S, ckpt_every=K)
            out["adam"] = {"steps": 50, "lr": 1e-2, "loss": "weighted variance of E_L",
                           "variance_first": hist[0][0], "variance_last": hist[-1][0],
                           "variance_min": min(h[0] for h in hist),
                           "theta_final": th.tolist(), "seconds": time.perf_counter() - t0}
    return out


def run_adjoint(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    out = measure_adjoint(args.steps, args.warmup, adam=args.adam)
    out.update({"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "data": "synthetic"})
    print(json.dumps(out), flush=True)


def measure_walk(name, steps, warmup, *, rank, ws, peaks, n_sm, threads=0, wpt=0,
                 e2e=False, fp64_moves=0):
    """One workload on the walk kernels: `steps` device-timed runs after `warmup`, L2
    flushed before each, clocks sampled.  Returns the fields of its JSON object (and the
    mixed E(t) of instance 0 for the FP64 comparison)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1703_08977_gb300 import gfk

    insts, n_moves = _workload(name, rank)
    n_walkers = sum(d["n_walkers"] for d in insts)
    trials = [(d["kind"], d["params"]) for d in insts]

    def descs(prec):
        return [gfk.InstanceDesc(n_walkers=d["n_walkers"], dt=d["dt"], e_trial=d["e_trial"],
                                 seed=d["seed"], state=d["state"], prec=prec,
                                 rng_stream=d["rng_stream"], walker_id0=d["walker_id0"],
                                 noise=d["noise"])
                for d in insts]

    ctx = gfk.Context(descs(gfk.GFK_PREC_MIXED), trials=trials)
    if threads and wpt:
        ctx.set_launch(threads, wpt)
        launch = (threads, wpt, None)
    else:
        launch = gfk.autotune_cached(ctx.handle, ctx.descs, trials, probe_steps=256)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB of L2
    stream = torch.cuda.current_stream()

    def device_step():
        ctx.reset()
        ctx.propagate(n_moves)

    for _ in range(warmup):
        device_step()
    torch.cuda.synchronize()

    # ---- timed region: `steps` device-resident runs, L2 flushed between them ----
    gfk.gfk_profile(ctx.handle, True)
    gfk.gfk_profile_read(ctx.handle, reset=True)
    gfk.gfk_kernel_count(ctx.handle, reset=True)
    clocks = Clocks(torch.cuda.current_device())
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    evs = []
    for _ in range(steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        device_step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    walk_ms, walk_launches, walk_ws = gfk.gfk_profile_read(ctx.handle, reset=True)
    kernels_timed = gfk.gfk_kernel_count(ctx.handle, reset=True)   # the library's own count
    gfk.gfk_profile(ctx.handle, False)
    if ws > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    walker_steps_per_step = n_walkers * n_moves
    out = {"value": walker_steps_per_step * ws * steps / (ms / 1e3), "unit": UNIT,
           "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
           "config": bench_config(name, rank),
           "launch": {"threads": launch[0], "walkers_per_thread": launch[1],
                      "chosen_by": "autotune" if launch[2] else "flags"},
           "gpu_launches": int(kernels_timed),
           "clocks": {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")}}
    sm_max = clk.get("sm_max_mhz") or 2070.0
    avg_launch_ms = walk_ms / max(1, walk_launches)
    ws_per_launch = walk_ws / max(1, walk_launches)
    out["roofline"], out["mufu"], out["issue"] = walk_rooflines(
        name, insts, avg_launch_ms, ws_per_launch, peaks, n_sm, sm_max, clk.get("sm_mhz"))

    e_mixed = None
    if e2e:
        # ---- end to end through the C ABI with host buffers (graph replay) ----
        cap = n_moves + 1
        e_host = [np.empty(cap) for _ in insts]
        lz_host = [np.empty(cap) for _ in insts]
        ess_host = [np.empty(cap) for _ in insts]
        h2d = sum(8 * len(p) for _, p in trials) + 1024 * len(insts)   # trials + instance table
        d2h = len(insts) * (3 * 8 * cap + 8)
        ctx.set_graph(True)
        ctx.reset()
        ctx.propagate(n_moves)              # capture once (outside the timing)
        torch.cuda.synchronize()
        n_e2e = max(1, steps // 2)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            gfk.gfk_reset(ctx.handle)
            for i, (k, p) in enumerate(trials):
                gfk.gfk_set_trial(ctx.handle, i, k, p)
            gfk.gfk_propagate(ctx.handle, n_moves)
            for i in range(len(insts)):
                gfk.gfk_energy(ctx.handle, i, cap=cap, out=(e_host[i], lz_host[i], ess_host[i]))
        e2e_s = (time.perf_counter() - t0) / n_e2e
        if ws > 1:
            # the slowest rank's wall clock, as for the device-timed figure
            t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        out["e2e"] = {"value": walker_steps_per_step * ws / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "path": "gfk_set_trial + gfk_propagate (CUDA-graph replay) + gfk_energy "
                              "into host arrays, wall clock"}
        e_mixed = e_host[0].copy()
        if ws > 1:
            # the one exchange step: merge the ranks' per-step sums of instance 0
            from paper_1703_08977_gb300 import distributed as gd
            merged = gd.merge_sums(ctx.sums(0))
            out["merged_E_final_all_ranks"] = float(
                gd.estimators(merged, insts[0]["n_walkers"] * ws)["E"][-1])
    ctx.close()

    if fp64_moves and rank == 0:
        # ---- the FP64 path on the same seeds, and the mixed path's energy error ----
        if e_mixed is None:
            with gfk.Context(descs(gfk.GFK_PREC_MIXED), trials=trials) as cm:
                cm.propagate(fp64_moves)
                e_mixed = cm.energy(0)["E"]
        c64 = gfk.Context(descs(gfk.GFK_PREC_FP64), trials=trials)
        c64.propagate(32)
        torch.cuda.synchronize()
        c64.reset()
        gfk.gfk_profile(c64.handle, True)
        gfk.gfk_profile_read(c64.handle, reset=True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c64.propagate(fp64_moves)
        b.record(stream)
        torch.cuda.synchronize()
        w64_ms, w64_l, w64_ws = gfk.gfk_profile_read(c64.handle, reset=True)
        fp64_ms = a.elapsed_time(b)
        fp64_value = n_walkers * fp64_moves / (fp64_ms / 1e3)
        e64 = c64.energy(0)["E"]
        c64.close()
        counts = _op_counts(insts)
        r64 = w64_ws / (w64_ms / 1e3)
        diff = e_mixed[: fp64_moves + 1] - e64
        tail = diff[len(diff) // 2:]
        out["fp64_path"] = {
            "value": fp64_value, "unit": UNIT, "moves": fp64_moves,
            "mixed_over_fp64": out["value"] / ws / fp64_value,
            "roofline": {"bound": "alu", "achieved": counts["flops"] * r64 / 1e12,
                         "peak": 2.0 * peaks["dfma"] / 1e12, "unit": "TFLOP/s",
                         "frac": counts["flops"] * r64 / (2.0 * peaks["dfma"]),
                         "kernel": "walk_fp64_kernel",
                         "peak_basis": "of measured: DFMA lane rate (gfk_measure_peak) x 2 flops",
                         "note": "FP64 library exp/log/sqrt/sin/cos run as instruction sequences "
                                 "on the FP64 pipe, beyond the algorithmic flops counted here"}}
        out["energy_error_vs_fp64"] = {
            "moves": fp64_moves, "max_abs_E_t": float(np.max(np.abs(diff))),
            "mean_E_t_second_half": float(np.mean(tail)), "final": float(diff[-1]),
            "note": "mixed minus FP64 path, same seeds and walkers; the FP64 path "
                    "matches the FP64 oracle to 1e-13 (tests)"}
    return out


EXTRA_WALKS = ("triplet", "batched", "bernoulli")


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = _dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measure_peaks()
    main_line = measure_walk(args.workload, args.steps, args.warmup, rank=rank, ws=ws,
                             peaks=peaks, n_sm=n_sm, threads=args.threads, wpt=args.wpt,
                             e2e=True,
                             fp64_moves=args.fp64_moves if args.workload in ("ground", "bernoulli")
                             else 0)
    out = None
    if rank == 0:
        out = {"metric": METRIC, "n_gpus": ws, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic"}
        out.update(main_line)
        out["measured_peaks_lane_ops_per_s"] = peaks
    extras = {}
    if ws == 1 and args.workload == "ground" and not args.no_extras:
        # the other workloads of the scope, each its own measurement (3 warm-up runs,
        # 3 timed runs, L2 flushed before each, clocks sampled)
        for name in EXTRA_WALKS:
            extras[name] = measure_walk(name, 3, 3, rank=rank, ws=ws, peaks=peaks, n_sm=n_sm)
        extras["adjoint"] = measure_adjoint(3, 3, adam=True)
    if rank == 0:
        if extras:
            out["workloads"] = extras
        if not args.no_cpu_baseline and ws == 1:
            # the oracle on the host cores: a single-GPU figure, not repeated
            # while the other ranks of a multi-GPU run wait
            out["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def profile_case(args):
    """A small case for ncu captures: the workloads' trial function of state
    --profile-state (default 0, the ground state), two launches of
    --profile-moves moves each (default 64) on --profile-walkers walkers (default
    2^22 mixed, 2^20 FP64; the state is larger than L2 either way), mixed path (or
    FP64 with --prec 0), Gaussian or Bernoulli noise (--noise)."""
    import torch
    from paper_1703_08977_gb300 import gfk, workloads as wl
    kind, params = wl.trial_for_state(args.profile_state)
    n = args.profile_walkers or (1 << 22 if args.prec == 1 else 1 << 20)
    dt = 1.0 / 900.0 if args.noise == 1 else 0.005
    d = gfk.InstanceDesc(n_walkers=n, dt=dt, e_trial=wl.E_T[args.profile_state], seed=SEED,
                         prec=args.prec, noise=args.noise, state=args.profile_state)
    launch = (args.threads or 128, args.wpt or 2) if args.prec == 1 else (128, 1)
    m = args.profile_moves
    if args.profile_grad >= 0:
        # the gradient instead: two gfk_grad calls of --profile-moves moves with
        # checkpoints every --profile-grad moves (0: the whole trajectory kept),
        # on the gradient workload's trial function
        theta = [2.0, 0.5, 0.5, 0.0, 0.0, 0.0, 0.0]
        with gfk.Context([d], trials=[(0, theta)], launch=launch) as ctx:
            for _ in range(2):
                loss, g = gfk.gfk_grad(ctx.handle, 0, 0, m, args.profile_grad)
        print(json.dumps({"profile_case": True, "gradient": True, "walkers": n, "moves": m,
                          "ckpt_every": args.profile_grad, "prec": args.prec, "loss": loss,
                          "grad": g.tolist()}))
        return
    with gfk.Context([d], trials=[(kind, params)], launch=launch) as ctx:
        ctx.propagate(m)
        ctx.propagate(m)
        torch.cuda.synchronize()
        e = ctx.energy(0)["E"]
    print(json.dumps({"profile_case": True, "walkers": n, "moves": 2 * m, "prec": args.prec,
                      "noise": args.noise, "state": args.profile_state, "launch": launch,
                      "E_final": float(e[-1])}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ground", choices=sorted(WORKLOADS))
    ap.add_argument("--threads", type=int, default=0, help="launch shape (0: autotune)")
    ap.add_argument("--wpt", type=int, default=0, help="walkers per thread (0: autotune)")
    ap.add_argument("--fp64-moves", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline workload only (skip the triplet, batched, Bernoulli and "
                         "adjoint measurements)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run the small ncu capture case instead of the benchmark")
    ap.add_argument("--prec", type=int, default=1, help="profile case: 1 mixed, 0 FP64")
    ap.add_argument("--noise", type=int, default=0, help="profile case: 0 Gaussian, 1 Bernoulli")
    ap.add_argument("--profile-walkers", type=int, default=0)
    ap.add_argument("--profile-moves", type=int, default=64)
    ap.add_argument("--profile-grad", type=int, default=-1,
                    help="profile case: run gfk_grad with this checkpoint interval (0: the "
                         "whole trajectory kept) instead of the walk")
    ap.add_argument("--profile-state", type=int, default=0, choices=(0, 1, 2),
                    help="profile case: trial function of state 0 (1^1S), 1 (2^3S), 2 (P_z)")
    ap.add_argument("--adam", action="store_true", help="adjoint workload: run 50 Adam steps")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
