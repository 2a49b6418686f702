#!/usr/bin/env python3
"""Benchmark of the GB300 lattice Boltzmann elasticity solver.

Workload (default): the single-large-lattice throughput case -- a 16384 x 16384
doubly periodic lattice, FP32 population storage, E~ = 1, nu = 0.3, body force
made of 16 seeded random Fourier modes (amplitudes N(0,1)/|k|^2, |k_x|, |k_y| <= 8).
One benchmark step is one pass of the whole hot path over that input: reset to
the zero state, 1000 fixed pseudo-time steps of the fused stream-collide kernel
with the fused steady-state residual every 100 steps, then the FP64
displacement / stress recovery.  The metric is MLUPS (million lattice-node
updates per second); the stream-collide kernel's achieved HBM bandwidth is
reported against the measured copy peak.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica on its own GPU (the
problem does not shard; replicas only).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "MLUPS and HBM GB/s (% of GB300 peak); solves/sec and p99 latency, batched vs plain"
FALLBACK_HBM_GBS = 6800.0
# Algorithmic bytes per node and stream-collide launch: 8 populations read + 8
# written + 2 force components read; FP16-shifted adds the two FP32
# first-moment carriers read and written.  A launch advances one step, or two
# (FP32 two-step kernel): bytes per lattice update = this / steps per launch.
# the wavefront kernel runs from this lattice width up (one strip of slots)
WAVE_MIN_NX = 256
BYTES_PER_LAUNCH_NODE = {"f64": 8 * 8 * 2 + 2 * 8, "f32": 8 * 4 * 2 + 2 * 4, "f16s": (8 * 2 + 2 * 4) * 2 + 2 * 4}
FORCE_SEED = 0x2208_14870
# FP64 storage runs its collision on the FP64 pipe: 42 FP64 instructions per
# lattice update (ncu: 28 DADD, 5 DMUL, 9 DFMA per node), i.e. 51 flops.
# Every FP64 instruction takes one slot of the pipe, whose nominal rate on
# GB300 is 1.25 TFLOP/s counting an FMA as 2 flops, i.e. 625 G instructions/s.
FP64_INSTR_PER_LUP = 42
FP64_FLOPS_PER_LUP = 51
FP64_PEAK_GINST = 625.0
# DRAM traffic per stream-collide launch from one ncu capture, keyed by dtype,
# steps per launch and schedule, with the hash of the kernel code it was taken
# on (null in the bench line once the code changes; comments do not count).
# Captured at 8192^2 with 256-row segments (profiles/k_wave_8192_dram_traffic.md):
# 33 strips of 256 slots and 32 segments, the same column-halo share (256/250
# per output column) and segment length as the 16384^2 launch, so a launch's
# traffic is 4x the capture's (nodes x4).  Mean of three launches.
NCU_TRAFFIC = {
    "f32_x4w": {"bytes_per_launch": 4 * (2.76050e9 + 2.10493e9), "kernel_hash": "fb0329a445f0d126",
                "ncu": {"case": "8192^2, 256-row segments, x4", "dram_read_per_launch": 4 * 2.76050e9,
                        "dram_write_per_launch": 4 * 2.10493e9, "algorithmic_per_launch": 72 * 16384 ** 2}},
    "f16s_x4w": {"bytes_per_launch": 4 * (2.20988e9 + 1.57011e9), "kernel_hash": "fb0329a445f0d126",
                 "ncu": {"case": "8192^2, 256-row segments, x4", "dram_read_per_launch": 4 * 2.20988e9,
                         "dram_write_per_launch": 4 * 1.57011e9, "algorithmic_per_launch": 56 * 16384 ** 2}},
}


def kernel_source(text: str) -> str:
    """The part of lbm_kernels.cuh that defines the stream-collide kernel
    (gather, stores, residual reduction, tile body, k_step)."""
    a = text.index("// Gather the pre-collision populations")
    b = text.index("// Solution fields of the current state")
    return text[a:b]


def code_only(text: str) -> str:
    """C/CUDA source without comments and with whitespace collapsed."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash(read=None) -> str:
    """Hash of the code (comments and layout ignored) the stream-collide
    kernels are built from: the per-node arithmetic (lbm_core.cuh), the part
    of lbm_kernels.cuh up to the solution-field recovery (layout, gather,
    stores, residual, the one-, two-, three-step and wavefront kernels), the
    launchers and the per-storage translation units.  `read(name)` returns a
    file's text (default: this tree)."""
    d = os.path.join(ROOT, "paper_2208_14870_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(d, name)) as fh:
                return fh.read()
    h = hashlib.sha256()
    for name in ("lbm_core.cuh", "lbm_kernels.cuh", "lbm_ops.cuh", "lbm_step_f32.cu", "lbm_step_f16s.cu",
                 "lbm_wave_f32.cu", "lbm_wave_f16s.cu"):
        text = read(name)
        if name == "lbm_kernels.cuh":
            text = text[:text.index("// Destinations of the five solution fields")]
        h.update(code_only(text).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax = float(row[2])
                power.append(float(row[3]))
            except ValueError:
                continue
            for name, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_aggregate(dist, elapsed_ms: float, units: float, device="cpu"):
    """Replicas only: each rank times its own copy of the workload.  Returns
    (max elapsed ms over ranks, sum of units over ranks); without a process
    group, the local values."""
    import torch
    if dist is None or not dist.is_initialized():
        return elapsed_ms, units
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def make_force(n: int):
    pw = W.random_force(n, n, n_modes=16, kmax=8, seed=FORCE_SEED)
    return W.random_force_grid(pw)


# ---------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------

def _oracle_replica(job):
    """One oracle replica (a process of its own): `reps` times `iters`
    pseudo-time steps plus field recovery on an m x m lattice with the
    benchmark's force recipe; all replicas start together at `barrier`.
    Returns the replica's compute seconds."""
    m, iters, reps, nu, barrier = job
    import oracle
    lam, mu = W.lame_2d(1.0, nu)
    rates = oracle.relaxation_rates(lam, mu)
    pw = W.random_force(m, m, n_modes=16, kmax=8, seed=FORCE_SEED)
    gx, gy = W.random_force_grid(pw)
    oracle.run(oracle.zero_state(m, m), gx, gy, rates, 1)      # load and warm the library
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    for _ in range(reps):
        f = oracle.run(oracle.zero_state(m, m), gx, gy, rates, iters)
        oracle.fields(f, gx, gy, rates)
    return time.perf_counter() - t0


_REPLICA_BARRIER = None


def _replica_init(barrier):
    global _REPLICA_BARRIER
    _REPLICA_BARRIER = barrier


def _replica_job(job):
    return _oracle_replica(job + (_REPLICA_BARRIER,))


def oracle_all_cores(m, iters, reps, nu):
    """The oracle as it is, one replica per host core (spawned processes,
    started together): aggregate lattice updates per second over the slowest
    replica's time.  Returns (MLUPS, cores, seconds)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ncores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(ncores)
    with ctx.Pool(ncores, initializer=_replica_init, initargs=(barrier,)) as pool:
        times = pool.map(_replica_job, [(m, iters, reps, nu)] * ncores, chunksize=1)
    dt = max(times)
    return ncores * m * m * iters * reps / dt / 1e6, ncores, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    m = args.ref_n
    iters = args.ref_iters
    # warm-up steps run in the replicas before their barrier; the timed steps
    # are args.steps repetitions of the bounded sample on every core at once
    mlups, cores, dt = oracle_all_cores(m, iters, args.steps, args.nu)
    sample = ("%dx%d lattice, same 16-mode force recipe, %d pseudo-time steps + field recovery "
              "per benchmark step, one oracle replica per host core (%d processes)" % (m, m, iters, cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample, "host": host_description()},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": "single large lattice throughput: %dx%d periodic D2Q8, %s storage, "
                        "16 random Fourier force modes, %d fixed steps/step" % (
                            args.n, args.n, args.dtype.upper(), args.iters),
            "nx": args.n, "ny": args.n, "iters_per_step": args.iters,
            "check_every": args.check_every, "E": 1.0, "nu": args.nu,
            "force": "16 modes, |kx|,|ky|<=8, amp N(0,1)/|k|^2, seed %#x" % FORCE_SEED,
            "l2": "inputs larger than L2: %.1f GB of populations and force read+written per launch, L2 129 MB" % (
                args.n * args.n * BYTES_PER_LAUNCH_NODE[args.dtype] / 1e9)}


def cpu_baseline(args):
    """The FP64 C oracle as it is on the host cores: one replica per core
    (the headline figure, cores = the replicas), and a single replica alone
    beside it."""
    import oracle
    oracle.build()
    lam, mu = W.lame_2d(1.0, args.nu)
    rates = oracle.relaxation_rates(lam, mu)
    m, it = args.ref_n, args.ref_iters
    pw = W.random_force(m, m, n_modes=16, kmax=8, seed=FORCE_SEED)
    gx, gy = W.random_force_grid(pw)
    t0 = time.perf_counter()
    oracle.run(oracle.zero_state(m, m), gx, gy, rates, it)
    dt1 = time.perf_counter() - t0
    mlups, cores, dt = oracle_all_cores(m, it, 1, args.nu)
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%dx%d lattice, same force recipe, %d steps + field recovery, FP64 C oracle, one "
                      "replica per host core started together (%.1f s)" % (m, m, it, dt),
            "single_core": {"value": m * m * it / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                            "sample": "%dx%d lattice, %d steps, one replica alone (%.1f s)" % (m, m, it, dt1)},
            "host": host_description()}


def host_description():
    """The host the CPU baseline ran on: logical cores and CPU model."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "cpu implementer") and not model:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return {"logical_cores": os.cpu_count(), "machine": platform.machine(), "cpu": model}


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def plan_plain(m, spl, wave=False):
    """Launch sizes of m plain steps as the library groups them: launches of
    spl steps (four only on the wavefront schedule, else three), a remainder
    of one avoided where possible (4 = 2 + 2, 5 = 3 + 2), then pairs, then
    single steps."""
    sizes = []
    big = 4 if spl >= 4 and wave else (3 if spl >= 3 else 0)
    if big:
        groups, r = divmod(m, big)
        if r == 1 and groups >= 1:
            groups, r = groups - 1, r + big
        sizes += [big] * groups
        m = r
        if big == 4 and m >= 3:
            sizes.append(3)
            m -= 3
    if spl >= 2:
        sizes += [2] * (m // 2)
        m %= 2
    return sizes + [1] * m


def check_launch_steps(w, spl, wave=False):
    """Steps of the launch that ends a residual window of w steps: a four-step
    wavefront launch (check on its last level) where the schedule runs four
    steps per launch, else a launch of at most two steps."""
    return 4 if (wave and spl >= 4 and w >= 4) else min(spl, 2, w)


def launches_per_iterate(iters, check_every, spl, wave=False):
    """Stream-collide launches of lbm_iterate_checked(iters, check_every) from
    step 0: each window is check_every - 1 plain steps grouped into launches of
    spl steps (the remainder in shorter ones) and ends with the check step,
    the last step of the window's last launch (check_launch_steps)."""
    def window(w):
        last = check_launch_steps(w, spl, wave)
        return len(plan_plain(w - last, spl, wave)) + 1
    total, left = 0, iters
    while left >= check_every:
        total += window(check_every)
        left -= check_every
    return total + len(plan_plain(left, spl, wave))


def time_variant(args, dtype, gx_d, gy_d, torch, P, nsteps, nwarm, events=True, spl=None, iters=None,
                 wave=None):
    """Device-resident timing of `nsteps` benchmark steps of `iters`
    pseudo-time steps each (default --iters); returns dict."""
    n = args.n
    iters = args.iters if iters is None else iters
    lam, mu = W.lame_2d(1.0, args.nu)
    lat = P.Lattice(n, n, lam, mu, dtype)
    if spl is not None:
        lat.steps_per_launch = spl
    if wave is not None and dtype != "f64":
        lat.wavefront = wave
    spl = lat.steps_per_launch
    wave_on = dtype != "f64" and lat.wavefront != 0 and n >= WAVE_MIN_NX
    stream = torch.cuda.current_stream()
    lat.set_stream(stream.cuda_stream)
    lat.set_force(gx_d, gy_d)
    out5 = torch.empty(5 * n * n, dtype=torch.float64, device="cuda")

    ce = args.check_every
    windows, rest = divmod(iters, ce)
    block, big = dominant_block(ce, spl, wave_on)
    nev = nsteps * windows

    def one_step(ev_a=None, ev_b=None, dom=None):
        # The same launches as lbm_iterate_checked(iters, check_every): per
        # window, its whole launches of the dominant kernel (plain, `big` steps
        # each) between two events, then the rest of the window with its
        # check; the library places checks by step index, so splitting the
        # call changes nothing.
        lat.reset()
        if ev_a is not None:
            ev_a.record(stream)
        for _ in range(windows):
            if dom is not None:
                dom[0].record(stream)
            P.lbm_iterate(lat.ctx, block)
            if dom is not None:
                dom[1].record(stream)
                dom = dom[2:]
            P.lbm_iterate_checked(lat.ctx, ce - block, ce, None)
        if rest:
            P.lbm_iterate_checked(lat.ctx, rest, ce, None)
        if ev_b is not None:
            ev_b.record(stream)
        lat.fields_device(out5)

    for _ in range(nwarm):
        one_step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nsteps)]
    devs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * nev)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i, (a, b) in enumerate(evs):
        one_step(a, b, devs[2 * i * windows: 2 * (i + 1) * windows])
    t_end.record(stream)
    torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    iter_ms = sum(a.elapsed_time(b) for a, b in evs)
    dom_ms = sum(devs[2 * k].elapsed_time(devs[2 * k + 1]) for k in range(nev))
    dom_launches = nev * (block // big)
    lat.close()
    del out5
    per_iter = launches_per_iterate(iters, args.check_every, spl, wave_on)
    checks = iters // args.check_every      # each adds one residual-finish launch
    return {"total_ms": total_ms, "iter_ms": iter_ms, "steps": nsteps, "spl": spl, "iters": iters,
            "step_launches": nsteps * per_iter, "launches": nsteps * (per_iter + checks + 1),
            "dom_ms": dom_ms, "dom_launches": dom_launches, "big": big, "wave": wave_on}


def fp64_peak(P):
    """The FP64 roofline denominator: the device's measured FP64 FMA rate
    (lbm_fp64_fma_rate), else the nominal rate."""
    try:
        return float(P.lbm_fp64_fma_rate()), ("measured: lbm_fp64_fma_rate (8 independent dependent-DFMA "
                                              "chains per thread, every SM full, CUDA events)")
    except Exception as e:  # noqa: BLE001
        return FP64_PEAK_GINST, "nominal GB300 FP64 rate (1.25 TFLOP/s with FMA = 2 flops); measurement failed: %s" % e


def dominant_block(check_every, spl, wave=False):
    """(steps, k): the first steps of a residual window, which the library
    runs as whole plain launches of k steps each, k the longest launch of the
    window (lbm_iterate_checked plans the window's check_every - 1 plain steps
    so; see plan_plain)."""
    sizes = plan_plain(check_every - check_launch_steps(check_every, spl, wave), spl, wave)
    if not sizes:
        return 0, spl
    big = sizes[0]
    return big * sum(1 for k in sizes if k == big), big


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    import paper_2208_14870_gb300 as P

    n = args.n
    gx, gy = make_force(n)
    gx_d = torch.from_numpy(gx).cuda()
    gy_d = torch.from_numpy(gy).cuda()
    peak, peak_kind = measured_peaks()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local if ws > 1 else torch.cuda.current_device())
    barrier()
    sampler.start()
    res = time_variant(args, args.dtype, gx_d, gy_d, torch, P, args.steps, args.warmup, spl=args.spl,
                       wave=args.wave)
    barrier()
    clocks = sampler.stop()
    total_ms, lups = replica_aggregate(dist if ws > 1 else None, res["total_ms"],
                                       float(n) * n * args.iters * args.steps, device="cuda")
    value = lups / (total_ms / 1e3) / 1e6
    spl = res["big"]          # steps per launch of the dominant kernel
    # the dominant kernel: plain launches of spl steps, timed by events around
    # them inside the timed region
    per_launch_s = res["dom_ms"] / 1e3 / res["dom_launches"]
    # a launch reads and writes the populations once and reads the force once,
    # whatever number of steps it advances
    bpl = BYTES_PER_LAUNCH_NODE[args.dtype] * n * n
    achieved = bpl / per_launch_s / 1e9
    tr = NCU_TRAFFIC.get("%s_x%d%s" % (args.dtype, spl, "w" if res["wave"] else ""))
    current = bool(tr) and tr.get("kernel_hash") == kernel_hash()
    traffic = tr["bytes_per_launch"] if current else None
    ncu_util = tr.get("ncu") if current else None

    variants = {}
    # the storage-type variants, the batched and the served workloads are
    # single-GPU measurements: taken at N = 1 only, so that a scaling run holds
    # its GPUs for the replicated throughput and end-to-end steps alone
    if not args.quick and ws == 1:
        for name in args.variants:
            mt = re.fullmatch(r"(f64|f32|f16s)(?:x(\d))?(w?)", name)
            if name == args.dtype or mt is None:
                continue
            dt, k, w = mt.groups()
            # "w": wavefront schedule; an explicit k without it: tile schedule
            r = time_variant(args, dt, gx_d, gy_d, torch, P, max(2, args.steps // 2), 2,
                             spl=int(k) if k else None,
                             iters=args.f64_iters if dt == "f64" else None,
                             wave=args.wave_rows if w else (0 if k else None))
            pl = r["dom_ms"] / 1e3 / r["dom_launches"]
            b = BYTES_PER_LAUNCH_NODE[dt] * n * n
            lups = float(n) * n * r["iters"] * r["steps"] / (r["total_ms"] / 1e3)
            variants[name] = {
                "value": lups / 1e6, "unit": "MLUPS", "ms_per_step": r["total_ms"] / r["steps"],
                "iters_per_step": r["iters"],
                "steps_per_launch": r["big"], "wavefront": r["wave"], "kernel_us": pl * 1e6,
                "achieved_gbs": b / pl / 1e9, "frac_of_measured_hbm": b / pl / 1e9 / peak,
                "bytes_per_lup": BYTES_PER_LAUNCH_NODE[dt] / r["big"]}
            if dt == "f64":
                # FP64 is bound by the FP64 pipe, not by HBM: FP64 instructions
                # per second over the device's measured FP64 FMA rate
                gi = FP64_INSTR_PER_LUP * n * n / pl / 1e9
                fpk, fkind = fp64_peak(P)
                variants[name]["roofline"] = {
                    "bound": "alu", "achieved": gi, "peak": fpk, "unit": "G FP64 instr/s",
                    "frac": gi / fpk, "peak_kind": fkind,
                    "fp64_instructions_per_lup": FP64_INSTR_PER_LUP, "flops_per_lup": FP64_FLOPS_PER_LUP,
                    "achieved_tflops": FP64_FLOPS_PER_LUP * n * n / pl / 1e12}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, gx, gy, torch, P, ws, dist if ws > 1 else None)
    del gx_d, gy_d
    torch.cuda.empty_cache()
    batched = None if (args.no_batched or args.quick or ws > 1) else run_batched(args, P)
    served = None if (args.no_served or args.quick or ws > 1) else run_served(args, P)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic (seeded random Fourier-mode body force)",
            "config": workload_config(args),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": ("k_wave<%s,%d> (%d fused stream-collide steps per launch, "
                                    "wavefront schedule)" % (args.dtype, spl, spl)) if res["wave"] else
                                   {1: "k_step<%s> (fused stream-collide)",
                                    2: "k_step2<%s> (two fused stream-collide steps per launch)",
                                    3: "k_step3<%s> (three fused stream-collide steps per launch)"}[spl]
                                   % args.dtype,
                         "kernel_us": per_launch_s * 1e6, "steps_per_launch": spl,
                         "bytes_per_launch_node": BYTES_PER_LAUNCH_NODE[args.dtype],
                         "bytes_per_lup": BYTES_PER_LAUNCH_NODE[args.dtype] / spl,
                         "peak_kind": peak_kind + " copy bandwidth",
                         "frac_of_nominal_8tbs": achieved / 8000.0,
                         # with several steps per launch the kernel moves fewer bytes per
                         # update than the HBM roofline of one step per launch allows for;
                         # the bandwidth that one-step schedule would need, and what ncu
                         # says binds the kernel instead
                         "one_step_equivalent_gbs": achieved * spl,
                         "one_step_equivalent_frac": achieved * spl / peak,
                         "ncu_utilisation": ncu_util},
            "clocks": clocks,
            "gpu_launches": res["launches"],
            "e2e": e2e,
            "variants": variants,
            "batched": batched,
            "served": served,
        }
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_e2e(args, gx, gy, torch, P, ws, dist):
    """Through the public API with host buffers: upload the force from pinned
    host memory, reset, iterate with residual checks, read displacement and
    stress back into pinned host memory -- every step.  With a pipeline of
    p > 1, p lattices on their own streams are driven by p host threads (step
    s on lattice s mod p) with copy-engine transfers (LBM_HOST_COPY), so one
    lattice's transfers overlap another's steps; every step still carries its
    own host-to-device and device-to-host copies."""
    import threading
    n = args.n
    pipe = max(1, args.e2e_pipeline)
    lam, mu = W.lame_2d(1.0, args.nu)
    hgx = torch.from_numpy(gx).pin_memory()
    hgy = torch.from_numpy(gy).pin_memory()
    lanes = []
    for k in range(pipe):
        lat = P.Lattice(n, n, lam, mu, args.dtype)
        stream = None
        if pipe > 1:
            stream = torch.cuda.Stream()
            lat.set_stream(stream.cuda_stream)
        lat.host_transfer = P.LBM_HOST_COPY if args.e2e_transfer == "copy" else P.LBM_HOST_DIRECT
        outs = [torch.empty(n * n, dtype=torch.float64).pin_memory() for _ in range(5)]
        lanes.append({"lat": lat, "stream": stream, "outs": outs, "res": np.zeros(5), "parts": np.zeros(4)})

    def step(lane):
        # every call returns after its work is done (the library synchronises
        # its stream), so the host clock between calls splits the step
        lat, outs, res = lane["lat"], lane["outs"], lane["res"]
        t = [time.perf_counter()]
        P.lbm_set_force(lat.ctx, hgx.data_ptr(), hgy.data_ptr())
        t.append(time.perf_counter())
        P.lbm_reset(lat.ctx)
        P.lbm_iterate_checked(lat.ctx, args.iters, args.check_every, res.ctypes.data)
        t.append(time.perf_counter())
        P.lbm_get_displacement(lat.ctx, outs[0].data_ptr(), outs[1].data_ptr())
        t.append(time.perf_counter())
        P.lbm_get_stress(lat.ctx, outs[2].data_ptr(), outs[3].data_ptr(), outs[4].data_ptr())
        t.append(time.perf_counter())
        lane["parts"][:] += np.diff(t)

    def run(nsteps):
        errors = []

        def lane_loop(k):
            try:
                for _ in range(k, nsteps, pipe):
                    step(lanes[k])
            except Exception as e:  # re-raised on the main thread
                errors.append(e)

        threads = [threading.Thread(target=lane_loop, args=(k,)) for k in range(pipe)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]

    run(args.e2e_warmup * pipe)
    torch.cuda.synchronize()
    for lane in lanes:
        lane["parts"][:] = 0.0
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    run(args.e2e_steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    t = torch.tensor([dt], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dt = float(t.item())
    parts = sum(lane["parts"] for lane in lanes) / args.e2e_steps
    for lane in lanes:
        lane["lat"].close()
    api = ("lbm_set_force(host) + lbm_reset + lbm_iterate_checked + "
           "lbm_get_displacement/lbm_get_stress(host)")
    if pipe > 1:
        api += ", %d lattices on their own streams, one host thread each" % pipe
    api += ", " + ("LBM_HOST_COPY (copy-engine transfers through device staging)" if args.e2e_transfer == "copy"
                   else "LBM_HOST_DIRECT (kernels read and write the pinned host arrays)")
    return {"value": float(n) * n * args.iters * args.e2e_steps * ws / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": 5 * n * n * 8 + 5 * 8,
            "steps": args.e2e_steps, "pipeline": pipe, "ms_per_step": dt / args.e2e_steps * 1e3,
            "api": api,
            "parts_ms": dict(zip(("set_force", "reset_iterate", "get_displacement", "get_stress"),
                                 (float(v) for v in parts * 1e3))),
            "parts_note": "host time per call and step, averaged over the steps"
                          + ("; calls of different lattices overlap" if pipe > 1 else "")}


# ---------------------------------------------------------------------------
# Batched and served workloads (time-boxed seeded subsets)
# ---------------------------------------------------------------------------

def plain_solve(P, p, tol, k, dtype="f32"):
    """One problem through the plain single-lattice API, host in and out."""
    gx, gy = W.random_force_grid(p.force)
    with P.Lattice(p.nx, p.ny, p.lam, p.mu, dtype) as lat:
        lat.set_force(gx, gy)
        st, it, r = lat.solve(tol, 10_000_000, k)
        lat.fields()
    return st, it


def run_sweep(args, P):
    """Convergence and stability sweep (the sinusoidal manufactured field at
    wavenumbers 1 and 4, E = 1, nu in {0, 0.2, 0.3, 0.4, 0.45}, N from 32 up):
    per storage type the relative error of u and sigma against the analytic
    field after ln(1/eps) / r steps (r = min(2 a^2 (mu + K), 0.05), a = 2 pi
    k / N: the decay rate of the forced mode, capped where the lattice's other
    modes decay slower), the observed order between successive N,
    and the device rate.  FP64 stops at --sweep-f64-max (its FP64-pipe rate
    makes N = 2048 minutes long)."""
    import torch
    eps = {"f64": 1e-13, "f32": 1e-8, "f16s": 1e-6}
    ns = [n for n in (32, 64, 128, 256, 512, 1024, 2048) if n <= args.sweep_max_n]
    rows = []
    stream = torch.cuda.current_stream()
    for dt in ("f64", "f32", "f16s"):
        for k in (1, 4):
            for nu in (0.0, 0.2, 0.3, 0.4, 0.45):
                prev = None
                for n in ns:
                    if dt == "f64" and n > args.sweep_f64_max:
                        continue
                    lam, mu = W.lame_2d(1.0, nu)
                    man = W.sinusoid(n, k, lam, mu)
                    gx, gy = man.force()
                    # the forced mode decays at r = 2 a^2 (mu + K) per step while
                    # that is small; the non-hydrodynamic modes at ~0.05 or faster
                    a = 2.0 * np.pi * k / n
                    r = min(2.0 * a * a * (2.0 * mu + lam), 0.05)
                    steps = int(np.ceil(np.log(1.0 / eps[dt]) / r))
                    with P.Lattice(n, n, lam, mu, dt) as lat:
                        lat.set_stream(stream.cuda_stream)
                        lat.set_force(gx, gy)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        lat.iterate(steps)
                        e1.record(stream)
                        got = lat.fields()
                        ms = e0.elapsed_time(e1)
                    ex = man.exact()
                    eu = max(float(np.max(np.abs(got[i] - ex[i]))) / float(np.max(np.abs(ex[i]))) for i in (0, 1))
                    es = max(float(np.max(np.abs(got[i] - ex[i]))) / float(np.max(np.abs(ex[i]))) for i in (2, 3, 4))
                    row = {"dtype": dt, "k": k, "nu": nu, "n": n, "steps": steps, "err_u": eu, "err_sigma": es,
                           "glups": float(n) * n * steps / (ms / 1e3) / 1e9,
                           "order_u": None if prev is None else float(np.log2(prev / eu))}
                    prev = eu
                    rows.append(row)
                    print("sweep %-4s k=%d nu=%.2f N=%5d steps=%8d err_u=%.3e err_sigma=%.3e order=%s" % (
                        dt, k, nu, n, steps, eu, es, "-" if row["order_u"] is None else "%.2f" % row["order_u"]),
                        file=sys.stderr, flush=True)
    return {"workload": "convergence and stability sweep: sinusoidal manufactured field, wavenumbers 1 and 4, "
                        "nu in {0, 0.2, 0.3, 0.4, 0.45}, N = 32..%d (FP64 to %d), error vs the analytic field "
                        "after ln(1/eps)/r steps" % (ns[-1], args.sweep_f64_max),
            "eps": eps, "rows": rows}


def run_jitter(args, P):
    """Rounding floor of the steady-state residual (reading c6b): a state
    iterated far past convergence (e^-40 of its slowest mode) keeps jittering;
    max|u^t - u^(t-w)| / max|u^t| over windows of w steps, three windows each,
    FP32 and FP16S, N = 64, 256, 1024, random 8-mode force, nu = 0.3."""
    rows = []
    for dtype in ("f32", "f16s"):
        for n in (64, 256, 1024):
            lam, mu = W.lame_2d(1.0, 0.3)
            pw = W.random_force(n, n, 8, 4, seed=7 + n)
            gx, gy = W.random_force_grid(pw)
            a = 2.0 * np.pi / n
            steps = int(40.0 / (mu * a * a))
            with P.Lattice(n, n, lam, mu, dtype) as lat:
                lat.set_force(gx, gy)
                lat.iterate(steps - steps % 100)
                for w in (100, 1000, 6000):
                    js = [float(lat.iterate_checked(2 * w, w)[0] * w) for _ in range(3)]
                    rows.append({"dtype": dtype, "n": n, "window": w, "jitter": js})
                    print("jitter %-4s N=%5d w=%5d %s" % (dtype, n, w, " ".join("%.2e" % j for j in js)),
                          file=sys.stderr, flush=True)
    return {"workload": "rounding floor of the residual: random 8-mode force, nu = 0.3, state iterated e^-40 "
                        "past convergence, max|u^t - u^(t-w)| / max|u^t| per window", "rows": rows}


def run_batched(args, P):
    """Batched stream (2048 problems, sides log-uniform in [32, 1024], nu in
    [0, 0.45], 8 random force modes, FP32, tol 1e-8): the problems whose longer
    side is at most --batched-cap, solved once in one arena and once one at a
    time through lbm_solve.  Both through the public API, host in and out."""
    probs = [p for p in W.batched_problems() if max(p.nx, p.ny) <= args.batched_cap]
    probs = probs[:args.batched_max]
    plist = []
    for p in probs:
        gx, gy = W.random_force_grid(p.force)
        plist.append((p.nx, p.ny, p.lam, p.mu, gx, gy))
    P.batch_solve(plist[:8], "f32", args.tol, args.check_every)          # warm-up
    t0 = time.perf_counter()
    res, rep = P.batch_solve(plist, "f32", args.tol, args.check_every)
    tb = time.perf_counter() - t0
    ok = sum(1 for r in res if r["status"] == 0)
    # the plain baseline: every plain_every-th problem of the same stream (an
    # unbiased sample of its size and parameter distribution), one at a time
    sample = probs[::args.batched_plain_every]
    t0 = time.perf_counter()
    iters = 0
    for p in sample:
        st, it = plain_solve(P, p, args.tol, args.check_every)
        iters += it
    tp = time.perf_counter() - t0
    return {"workload": "batched stream of independent problems (seed %#x), %d problems with max side <= %d, FP32, "
                        "tol %g, residual every %d steps" % (0x5EED_BA7C4ED, len(probs),
                                                             args.batched_cap, args.tol,
                                                             args.check_every),
            "max_side": max(max(p.nx, p.ny) for p in probs),
            "problems": len(probs), "converged": ok,
            "solves_per_s": len(probs) / tb, "plain_solves_per_s": len(sample) / tp,
            "plain_sample": "every %d-th problem of the same stream (%d of %d), solved one at a time "
                            "through lbm_solve" % (args.batched_plain_every, len(sample), len(probs)),
            "speedup_vs_plain": (len(probs) / tb) / (len(sample) / tp), "wall_s": tb, "plain_wall_s": tp,
            "lattice_updates": rep["lattice_updates"],
            "glups_device": rep["lattice_updates"] / (rep["device_ms"] / 1e3) / 1e9,
            "tile_v": rep["tile_v"], "chunks": rep["chunks"], "blocks": rep["blocks"]}


def run_served(args, P):
    """Served stream (Poisson arrivals, sides log-uniform in [64, 4096], nu in
    [0, 0.45], 8 random force modes, tol 1e-8, FP32 or FP16-shifted per request,
    HBM budget 150 GB): the first --served-max requests with max side <= --served-cap,
    arriving at --served-rate requests/s, through lbm_server_*; compared with a
    single-server queue of plain lbm_solve calls on the same requests."""
    import threading
    budget = int(args.served_budget_gb * 1e9)
    stream = W.served_requests(rate_hz=args.served_rate)
    picked = [i for i, r in enumerate(stream) if max(r.nx, r.ny) <= args.served_cap]
    picked = picked[:args.served_max]
    reqs = [stream[i] for i in picked]
    # Thinning a Poisson stream by the side cap keeps it Poisson at rate
    # rate * p; rescaling its clock by p restores the stated arrival rate.
    p_keep = len(picked) / float(picked[-1] + 1)
    t_first = reqs[0].arrival
    for r in reqs:
        r.arrival = t_first + (r.arrival - t_first) * p_keep
    forces = [W.random_force_grid(r.force) for r in reqs]
    tickets = [None] * len(reqs)
    with P.Server(budget, check_every=args.check_every) as srv:
        start = time.perf_counter()

        def feeder():
            for i, r in enumerate(reqs):
                delay = (r.arrival - t_first) - (time.perf_counter() - start)
                if delay > 0:
                    time.sleep(delay)
                tickets[i] = srv.submit(r.nx, r.ny, r.lam, r.mu, forces[i][0], forces[i][1],
                                        dtype=r.dtype, tol=args.tol)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        statuses = [srv.wait(t, 3600.0, fields=False)["status"] for t in tickets]
        st = srv.stats()
    # plain: each request alone through lbm_solve, served first-come first-served
    service = []
    for r in reqs:
        t0 = time.perf_counter()
        plain_solve(P, r, args.tol, args.check_every, r.dtype)
        service.append(time.perf_counter() - t0)
    done, lat = 0.0, []
    for r, s in zip(reqs, service):
        arr = r.arrival - t_first
        done = max(done, arr) + s
        lat.append((done - arr) * 1e3)
    lat = np.array(lat)
    return {"workload": "served stream of solve requests (seed %#x): first %d requests with max side <= %d, "
                        "Poisson arrivals at %g req/s, tol %g, FP32/FP16S per request, "
                        "HBM budget %g GB (each storage type's arena half of it)" % (
                            0x5E4FED, len(reqs), args.served_cap, args.served_rate, args.tol,
                            args.served_budget_gb),
            "requests": len(reqs), "converged": statuses.count(0),
            "max_side": max(max(r.nx, r.ny) for r in reqs),
            "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"], "p95_ms": st["p95_ms"],
            "p99_ms": st["p99_ms"], "peak_running": st["peak_running"],
            "budget_bytes": budget, "peak_resident_bytes": st["peak_resident_bytes"],
            "memory_waits": st["memory_waits"],
            "device_s": st["device_ms"] / 1e3, "chunks": st["chunks"], "tile_v": st["tile_v"],
            "lattice_updates": st["lattice_updates"],
            "glups_device": st["lattice_updates"] / max(st["device_ms"], 1e-9) / 1e6,
            "plain_solves_per_s": len(reqs) / (done - 0.0) if done > 0 else None,
            "plain_p50_ms": float(np.percentile(lat, 50)), "plain_p95_ms": float(np.percentile(lat, 95)),
            "plain_p99_ms": float(np.percentile(lat, 99)),
            "plain_service_s": float(sum(service))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--dtype", default="f32", choices=["f64", "f32", "f16s"])
    ap.add_argument("--nu", type=float, default=0.3)
    ap.add_argument("--spl", type=int, default=None,
                    help="steps per stream-collide launch of the main line (default: the library's choice)")
    ap.add_argument("--wave", type=int, default=None,
                    help="wavefront segment rows of the main line (0: tile schedule, -1: automatic; "
                         "default: the library's choice)")
    ap.add_argument("--wave-rows", type=int, default=-1,
                    help="wavefront segment rows of the variants with a 'w' suffix (-1: automatic)")
    ap.add_argument("--f64-iters", type=int, default=100,
                    help="pseudo-time steps per benchmark step of the FP64 variant")
    ap.add_argument("--variants", nargs="*",
                    default=["f16s", "f32x3", "f32x2", "f32x1", "f16sx1", "f64"],
                    help="extra storage variants; a suffix xK fixes K steps per launch on the tile "
                         "schedule, xKw on the wavefront schedule")
    ap.add_argument("--quick", action="store_true", help="skip the extra dtype variants")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--e2e-pipeline", type=int, default=1,
                    help="lattices solved side by side in the end-to-end measurement (1: one at a time)")
    ap.add_argument("--e2e-transfer", choices=("copy", "direct"), default="direct",
                    help="host transfers of the end-to-end measurement (lbm_set_host_transfer)")
    ap.add_argument("--e2e-warmup", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-n", type=int, default=1024)
    ap.add_argument("--ref-iters", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-cap", type=int, default=1024,
                    help="longest side of the batched problems kept (1024: the whole stream)")
    ap.add_argument("--batched-max", type=int, default=2048)
    ap.add_argument("--batched-plain-every", type=int, default=4,
                    help="the plain one-at-a-time baseline solves every k-th problem of the batch")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-cap", type=int, default=2048)
    ap.add_argument("--served-max", type=int, default=100)
    ap.add_argument("--served-rate", type=float, default=20.0)
    ap.add_argument("--served-budget-gb", type=float, default=4.0,
                    help="HBM budget of the server (small enough that admission waits on memory)")
    ap.add_argument("--sweep-max-n", type=int, default=2048)
    ap.add_argument("--sweep-f64-max", type=int, default=512)
    ap.add_argument("--only", choices=["batched", "served", "sweep", "jitter"], default=None,
                    help="run one secondary workload alone and print its JSON")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    ws, rank, local = dist_setup()
    if args.only:
        import torch
        torch.cuda.set_device(local)
        import paper_2208_14870_gb300 as P
        out = {"batched": run_batched, "served": run_served, "sweep": run_sweep,
               "jitter": run_jitter}[args.only](args, P)
        print(json.dumps({"only": args.only, **out}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
