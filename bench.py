#!/usr/bin/env python3
"""Benchmark of the Caputo L1 time-marching solve (libftoep) on synthetic workloads.

Default workload: the batched mixed-precision solve -- 512 independent problems with
N log-uniform in [2^10, 2^17], M log-uniform in [63, 2047], gamma in (0.1, 0.95) u
(1.05, 1.9), random separable sources (seed 1234) -- compared with the plain double
solve of the same batch.  One step = one full solve of every problem (sine transform,
half-split Toeplitz solve of every mode, inverse transform, residual and one correction
sweep) with inputs resident in HBM.  --workload diffusion|wave|scalar time the single
problems (gamma 0.7, M 1023, N 65536 double; gamma 1.5, M 4095, N 262144 mixed; the scalar
ODE, N 1024).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle (plain
O(M N^2) direct time marching) on a bounded time prefix of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M·N unknowns/sec at ≤1e-6 rel err: mixed-precision batched vs plain FP64"
SOLVER_NAMES = {1: "half-split", 2: "inverse series"}
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (profiling recipe); probe measured 1.19 (DFMA loop)
# FP32 from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["diffusion", "wave", "wave_cn", "scalar", "batched", "twosided", "advection", "gmres",
                             "adjoint"])
    ap.add_argument("--nprob", type=int, default=512, help="batched workload: number of problems")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="default: fp64 for diffusion/scalar, mixed for wave")
    ap.add_argument("--no-compare", action="store_true", help="skip the mixed-precision comparison run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-singles", action="store_true", help="batched: skip the single-problem lines")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) leg (profiling runs)")
    ap.add_argument("--no-tune", action="store_true", help="batched: library default tuning instead of the autotuner's")
    ap.add_argument("--scheduler", type=int, default=0, choices=[0, 1, 2],
                    help="0 library (or tuned) choice, 1 per-level launches, 2 persistent chain")
    ap.add_argument("--solver", type=int, default=0, choices=[0, 1, 2],
                    help="0 library (or tuned) choice, 1 half-split, 2 inverse series")
    ap.add_argument("--M", type=int, default=None, help="override the workload's interior points (profiling cases)")
    ap.add_argument("--N", type=int, default=None, help="override the workload's time steps (profiling cases)")
    return ap.parse_args()


def workload(name, nprob=512, M=None, N=None):
    from paper_1710_11593_gb300 import workloads as wl
    if name == "batched":
        probs = wl.config_batched(nprob=nprob)
        return probs, f"batched{nprob}_N2^10-2^17_M63-2047_seed1234"
    if name == "diffusion":
        p = wl.config_diffusion(M=M or 1023, N=N or 65536)
        return p, f"diffusion_g0.7_M{p.M}_N{p.N}"
    if name == "wave":
        p = wl.config_wave(M=M or 4095, N=N or 262144)
        return p, f"wave_g1.5_M{p.M}_N{p.N}"
    if name == "wave_cn":  # config 3's problem with the Crank-Nicolson average of the spatial term
        p = wl.config_wave(M=M or 4095, N=N or 262144)
        p.kind = 2
        return p, f"wave_cn_g1.5_M{p.M}_N{p.N}"
    p = wl.config_scalar(N=N or 1024)
    return p, f"scalar_g0.5_N{p.N}"


# ----------------------------------------------------------------------------- flops model

def block_flops_per_unknown(B, L, Sf):
    """Nominal flops per unknown of one in-block solve: leaf substitution (L), direct
    levels L <= s < Sf (s each), FFT levels Sf <= s < B (5 log2(2s) + 3 each)."""
    f = float(L)
    s = L
    while s < B:
        f += s if s < Sf else 5 * math.log2(2 * s) + 3
        s *= 2
    return f


def tuning_of(precision, Np):
    B = min(4096, Np)
    L = min(16, B)
    return B, L, 64


def flop_model(p, precision):
    """Nominal flops of one solve per kernel class (5 n log2 n per complex FFT of length n,
    6 per complex product, 2 per multiply-add), following the schedule of the library."""
    return work_model(p, precision)[0]


def work_model(p, precision, solver=1):
    """(flops, bytes) of one solve per kernel class.  Bytes are the compulsory HBM bytes
    of each class's algorithm: every array the class reads or writes crosses HBM once
    (z pairs 8 B per complex float / 16 B double, fields 8 B per double, 4 B per float);
    the four-step scratch round trips are not counted (they are the implementation's).
    solver 2 (inverse series): each solve is one convolution of length n = 2 Np per pair
    (two FFTs, the partner product: 8 flops per point), reading z and the pair's packed
    spectrum (n complex) and writing z; the half-split classes are then empty."""
    Np = 16
    while Np < p.N:
        Np *= 2
    B, L, Sf = tuning_of(precision, Np)
    P = (p.M + 1) // 2
    nblk = -(-p.N // B)
    ncols = nblk * B
    nsolve = 1 if precision == "fp64" else 2
    zb = 16 if precision == "fp64" else 8  # bytes per complex of the solve
    inverse = inverse_b = 0.0
    if solver == 2:
        n = 2 * Np
        inverse = nsolve * P * (2 * 5 * n * math.log2(n) + 8 * n)
        inverse_b = nsolve * P * (2 * Np * zb + n * zb)
        nblk = 1  # no block solves or cross-block levels in the flops below
    # block solve = causal convolution with the block inverse: FFT and inverse FFT of length
    # 2B per pair plus two complex products per point; reads z, writes z, reads the
    # Hermitian-packed C1/C2 array (2B complex per pair)
    block = 0.0 if solver == 2 else nsolve * nblk * (2 * P * B) * (10 * math.log2(2 * B) + 14)
    block_b = 0.0 if solver == 2 else nsolve * nblk * P * (2 * B * zb + (2 * B) * zb)
    conv_smem = conv_4 = 0.0
    smem_b = four_b = 0.0
    nsmem = 4096 if precision == "fp64" else 8192
    for v in range(1, nblk):
        s = B << ((v & -v).bit_length() - 1)
        fl = P * (20 * s * math.log2(2 * s) + 12 * s)
        by = P * 3 * s * zb  # input half, output half read and written
        if 2 * s <= nsmem:
            conv_smem += fl
            smem_b += by
        else:
            conv_4 += fl
            four_b += by
    conv_smem *= nsolve
    conv_4 *= nsolve
    smem_b *= nsolve
    four_b *= nsolve
    sine = sine_b = 0.0
    if p.space == 1:
        K2 = 2 * (p.M + 1)
        sine = 2 * nsolve * (ncols / 2) * 5 * K2 * math.log2(K2)
        fb = 8  # double field in, out (fp64) / f double, v float, r float (mixed)
        sine_b = nsolve * (p.M * p.N * (fb + (fb if precision == "fp64" else 4)) + 2 * P * ncols * zb)
    flops = {"block_solve": block, "conv_smem": conv_smem, "conv_fourstep": conv_4, "sine": sine, "inverse": inverse}
    byts = {"block_solve": block_b, "conv_smem": smem_b, "conv_fourstep": four_b, "sine": sine_b,
            "inverse": inverse_b}
    # the persistent per-pair solve runs the block solves and every cross-block level
    flops["chain"] = block + conv_smem + conv_4
    byts["chain"] = block_b + smem_b + four_b
    if precision == "mixed":  # residual product of length 2Np in float-float, residual kernel
        n = 2 * Np
        flops["residual"] = P * (10 * n * math.log2(n) + 6 * n)
        byts["residual"] = P * n * 16 * 2 + p.M * p.N * (8 + 8 + 4)
    return flops, byts


# DRAM bytes (read + write) of the float chain kernel per unknown it solves, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of a launch of the 32-problem batch of
# the same generator (5.92e8 unknowns in one group: 42.6 GB per launch; profiles/
# chain_solve_kernel.md); a launch's traffic grows with the unknowns it solves.
CHAIN_FLOAT_DRAM_BYTES_PER_UNKNOWN = 42.66e9 / 591616893


def chain_roofline(flops, byts, prof, precision, units=None):
    """Roofline of the persistent per-pair solve of a batched plan from its own event time:
    a chain launch runs alone on the GPU (every per-problem phase before it has joined, the
    ones after it wait for it), in the timed solves as in the instrumented one, so its
    event time is its time in a timed step."""
    ms, ops, launches = prof.get("chain", (0.0, 0, 0))
    if ms <= 0 or flops.get("chain", 0.0) <= 0:
        return None
    sec = ms * 1e-3
    if precision == "mixed":
        peak, what = FP32_PEAK_TFLOPS, "FP32 from unit counts: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"
    else:
        peak, what = FP64_PEAK_TFLOPS, "FP64 nominal 1.25 TFLOP/s (DFMA probe: 1.19)"
    alu = flops["chain"] / sec / 1e12
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
    hbm = byts["chain"] / sec / 1e9
    alu_obj = {"bound": "alu", "achieved": alu, "peak": peak, "unit": "TFLOP/s", "frac": alu / peak,
               "peak_note": what}
    hbm_obj = {"bound": "hbm", "achieved": hbm, "peak": hbm_peak, "unit": "GB/s", "frac": hbm / hbm_peak,
               "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    main, other = (alu_obj, hbm_obj) if alu_obj["frac"] >= hbm_obj["frac"] else (hbm_obj, alu_obj)
    out = dict(main)
    traffic = None
    if precision == "mixed" and units and launches:
        # every unknown passes through two chain launches per step (first solve, correction)
        traffic = CHAIN_FLOAT_DRAM_BYTES_PER_UNKNOWN * 2 * units / launches
    out.update({"kernel_class": "chain", "kernel": "chain_solve_kernel", "class_ms_per_step": ms,
                "launches_per_step": launches, "per_launch_ms": ms / max(1, launches), "traffic": traffic,
                "traffic_note": "dram bytes per launch: a 32-problem ncu capture scaled by the unknowns per launch"
                if traffic else None,
                "other_bound": other,
                "note": "flops: 5 n log2 n per complex FFT of length n, 6 per complex product (block solves and "
                        "every cross-block level of both solves); bytes: compulsory HBM bytes of those steps; "
                        "time: CUDA events around each chain launch (it runs alone)"})
    return out


def roofline_of(flops, byts, prof, ms_per_step, precision):
    """Roofline of the dominant kernel class.  The class times come from one instrumented
    solve in which every kernel runs on one stream (no overlap), so the class's share of
    that solve times ms_per_step is its time inside a timed step; achieved = the class's
    algorithmic flops (bytes) per step over that time, against the ALU peak of its
    arithmetic (bytes: the measured HBM copy bandwidth).  The binding one (larger
    fraction) is reported, the other beside it."""
    total = sum(v[0] for v in prof.values())
    name = max(prof, key=lambda k: prof[k][0])
    ms, ops, launches = prof[name]
    if name not in flops or ms <= 0 or total <= 0 or flops[name] <= 0:
        return None
    share = ms / total
    sec = share * ms_per_step * 1e-3
    if precision == "mixed":  # float and float-float arithmetic: FP32 instructions
        peak, what = FP32_PEAK_TFLOPS, "FP32 from unit counts: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"
    else:
        peak, what = FP64_PEAK_TFLOPS, "FP64 nominal 1.25 TFLOP/s (DFMA probe: 1.19)"
    alu = flops[name] / sec / 1e12
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
    hbm = byts.get(name, 0.0) / sec / 1e9
    alu_frac, hbm_frac = alu / peak, hbm / hbm_peak
    alu_obj = {"bound": "alu", "achieved": alu, "peak": peak, "unit": "TFLOP/s", "frac": alu_frac,
               "peak_note": what}
    hbm_obj = {"bound": "hbm", "achieved": hbm, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac,
               "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    main, other = (alu_obj, hbm_obj) if alu_frac >= hbm_frac else (hbm_obj, alu_obj)
    out = dict(main)
    out.update({"kernel_class": name, "class_share": share, "class_ms_per_step": share * ms_per_step,
                "launches_per_step": launches, "per_launch_ms": share * ms_per_step / max(1, launches),
                "traffic": None, "other_bound": other,
                "note": "flops: 5 n log2 n per complex FFT of length n, 6 per complex product; bytes: "
                        "compulsory HBM bytes of the class (no four-step scratch); class time = its share of "
                        "one single-stream instrumented solve x ms_per_step"})
    return out


def class_profile(plan, f, u):
    """Kernel-class event times of one instrumented solve (every kernel on one stream)."""
    plan.profile(True)
    plan.solve(f, u)
    prof = plan.profile_read()
    plan.profile(False)
    return prof


class Ranks:
    """Rank context of one bench process (one process per GPU, launched by torchrun).
    The workload is a replica per rank (no data-path collective): the value is the units of
    all ranks over the slowest rank's time (weak scaling)."""

    def __init__(self, backend="nccl", device="cuda"):
        import torch.distributed as dist
        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        if self.world > 1 and not dist.is_initialized():
            dist.init_process_group(backend)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, x):
        """Largest x over the ranks (every rank gets it)."""
        if self.world == 1:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def value(self, units_per_rank, ms_max):
        """Whole-job throughput: units of all ranks / slowest rank's time."""
        return self.world * units_per_rank / (ms_max * 1e-3)

    def close(self):
        if self.world > 1 and self.dist.is_initialized():
            self.dist.destroy_process_group()


def host_memory_bytes():
    """Physical memory of the host, or the container's memory limit if smaller."""
    total = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            with open(path) as fh:
                v = fh.read().strip()
            if v.isdigit():
                total = min(total, int(v))
        except OSError:
            pass
    return total


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- oracle timing

def time_oracle(p, nprefix, reps=1):
    """Time the CPU oracle on the first nprefix steps of the workload (same tau)."""
    from oracle import oracle as orc
    from paper_1710_11593_gb300 import workloads as wl
    f = wl.materialize(p.source, p.kind, p.N, p.M, t=wl.time_points(p.kind, p.N, p.T)[:nprefix])
    T = p.T * nprefix / p.N
    th = orc.default_threads()
    t0 = time.perf_counter()
    for _ in range(reps):
        orc.march(p.kind, p.space, p.gamma, f, T=T, L=p.L, lam=p.lam, nthreads=th)
    dt = (time.perf_counter() - t0) / reps
    return p.M * nprefix / dt, dt, th


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p, wname = workload(args.workload, args.nprob, M=args.M, N=args.N)
    if isinstance(p, list):
        # batched workload: each step is the oracle on the first min(N, 512) levels of the
        # first 8 problems (all their points)
        sample_probs = [(q, min(q.N, 512)) for q in p[:8]]
        sample = "first min(N,512) levels of the first 8 problems (same tau), all points; O(M N^2) direct marching"
        config = {"workload": wname, "nprob": len(p), "precision": "fp64"}
    else:
        nprefix = min(p.N, 1024 if p.M > 1 else p.N)
        sample_probs = [(p, nprefix)]
        sample = f"first {nprefix} of {p.N} time steps, all {p.M} points (same tau); O(M N^2) direct marching"
        config = {"workload": wname, "M": p.M, "N": p.N, "gamma": p.gamma, "precision": "fp64"}
    units = sum(q.M * n for q, n in sample_probs)
    for _ in range(args.warmup):
        for q, n in sample_probs:
            time_oracle(q, n)
    tot, th = 0.0, 1
    for _ in range(args.steps):
        for q, n in sample_probs:
            _, dts, th = time_oracle(q, n)
            tot += dts
    dt = tot / args.steps
    v = units / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
           "cpu_baseline": {"value": v, "unit": "unknowns/s", "cores": th, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ----------------------------------------------------------------------------- GPU arm

def batch_field(probs, device="cuda"):
    import torch
    from paper_1710_11593_gb300 import workloads as wl
    units = sum(p.M * p.N for p in probs)
    f = torch.empty(units, dtype=torch.float64, device=device)
    off = 0
    for p in probs:
        n = p.M * p.N
        wl.materialize_torch(p.source, p.kind, p.N, p.M, device=device, out=f[off:off + n].view(p.M, p.N))
        off += n
    return f


def timed(plan, f, u, steps, warmup, rk, local, clocks=True):
    """Warm-up solves, then `steps` solves between CUDA events on the plan's stream (the
    current torch stream), barrier and synchronize on both sides.  Returns (ms per step,
    kernels launched per step, clock record)."""
    import torch
    for _ in range(warmup):
        plan.solve(f, u)
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if clocks else None
    plan.profile(False)  # resets the launch counters; no per-launch events in the timed steps
    rk.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.solve(f, u)
    e1.record()
    torch.cuda.synchronize()
    rk.barrier()
    clk = sampler.stop() if sampler else None
    launches = sum(v[2] for v in plan.profile_read().values()) / max(1, steps)
    return e0.elapsed_time(e1) / steps, launches, clk


def oracle_prefix_error(p, u, n0):
    """Relative error (2-norm and max over max) of the first n0 levels of the GPU field u
    [M][N] against the oracle's solve of the n0-level problem with the same tau."""
    import numpy as np
    from oracle import oracle as orc
    from paper_1710_11593_gb300 import workloads as wl
    fpre = wl.materialize(p.source, p.kind, p.N, p.M, t=wl.time_points(p.kind, p.N, p.T)[:n0])
    ref = orc.march(p.kind, p.space, p.gamma, fpre, T=p.T * n0 / p.N, L=p.L, lam=p.lam)
    got = u[:, :n0].cpu().numpy()
    return float(max(np.linalg.norm(got - ref) / np.linalg.norm(ref), np.max(np.abs(got - ref)) / np.max(np.abs(ref))))


def run_single(name, precision, steps, warmup, rk, local, tuning=None):
    """One single-problem workload: timed solves, class roofline, error against the oracle on
    a 1024-level prefix."""
    import torch
    from paper_1710_11593_gb300 import ftoep, workloads as wl
    p, wname = workload(name)
    prec = ftoep.FP64 if precision == "fp64" else ftoep.MIXED
    spec = ftoep.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec, lam=p.lam)
    f = wl.materialize_torch(p.source, p.kind, p.N, p.M, device="cuda")
    u = torch.empty_like(f)
    with ftoep.Plan([spec], tuning=tuning) as plan:
        ms, launches, _ = timed(plan, f, u, steps, warmup, rk, local, clocks=False)
        prof = class_profile(plan, f, u)
        plan.solve(f, u)
        plan.sync()
        solver = plan.solver(0)
    ms = rk.max(ms)
    fl, by = work_model(p, precision, solver)
    out = {"workload": wname, "precision": precision, "ms_per_step": ms, "value": p.M * p.N / (ms * 1e-3),
           "unit": "unknowns/s", "gpu_launches": launches, "solver": SOLVER_NAMES[solver],
           "roofline": roofline_of(fl, by, prof, ms, precision),
           "kernel_time_share": {k: v[0] / max(1e-9, sum(x[0] for x in prof.values())) for k, v in prof.items()},
           "rel_err_vs_oracle_prefix": oracle_prefix_error(p, u, min(p.N, 1024)),
           "oracle_prefix_levels": min(p.N, 1024)}
    del f, u
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    """Config-4 workload: all problems in one plan (chain schedule: groups of problems, one
    persistent launch per solve and group)."""
    import torch
    from paper_1710_11593_gb300 import ftoep

    rk = Ranks()
    world, rank, local = rk.world, rk.rank, rk.local
    torch.cuda.set_device(local)
    ftoep.load()
    probs, wname = workload("batched", args.nprob)
    precision = args.precision or "mixed"
    prec = ftoep.FP64 if precision == "fp64" else ftoep.MIXED
    specs = [ftoep.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in probs]
    units = sum(p.M * p.N for p in probs)
    f = batch_field(probs)
    u = torch.empty_like(f)
    # the autotuner's choice for this batch: the user's cache or the table shipped with the
    # package (written by paper_1710_11593_gb300/tune_table.py on a GB300), else a search
    tuning, cached = (None, None) if args.no_tune else ftoep.autotune_cached(specs)
    if args.scheduler or args.solver:  # explicit choices over the tuned ones
        tuning = dict(tuning or {})
        tuning.update({k: v for k, v in (("scheduler", args.scheduler), ("solver", args.solver)) if v})
    plan = ftoep.Plan(specs, tuning=tuning)
    ms, launches, clk = timed(plan, f, u, args.steps, args.warmup, rk, local)
    prof = class_profile(plan, f, u)
    ms = rk.max(ms)
    value = rk.value(units, ms)
    busy = sum(x[0] for x in prof.values())
    shares = {k: v[0] / max(1e-9, busy) for k, v in prof.items()}
    fl, by = {}, {}
    solvers = [plan.solver(i) for i in range(len(probs))]
    for p, sv in zip(probs, solvers):
        f1, b1 = work_model(p, precision, sv)
        for k in f1:
            fl[k] = fl.get(k, 0.0) + f1[k]
            by[k] = by.get(k, 0.0) + b1[k]
    roof = chain_roofline(fl, by, prof, precision, units) or roofline_of(fl, by, prof, ms, precision)
    # end to end through host buffers (pinned), copies inside the call.  All ranks of a node
    # share its host memory: the pinned buffers of all ranks are kept within 3/4 of it, and
    # when the whole batch does not fit the end-to-end step covers a prefix of the problems
    e2e = None
    fh, freed = None, False
    try:
        if args.no_e2e:
            raise ValueError("skipped (--no-e2e)")
        budget = 0.75 * host_memory_bytes() / max(1, world)
        k, e_units = len(probs), units
        while k > 1 and 2 * 8 * e_units > budget:
            k -= 1
            e_units -= probs[k].M * probs[k].N
        if k < len(probs):  # free the full plan's workspace before the sample's
            plan.close()
            plan = None
        fh = f[:e_units].cpu().pin_memory()
        uh = torch.empty_like(fh).pin_memory()
        # the host-buffer solve needs no device copy of the caller's fields: free them, so
        # that the plan can keep its own device copies (f in once, u out once per solve)
        del f, u
        freed = True
        torch.cuda.empty_cache()
        eplan = plan if plan is not None else ftoep.Plan(specs[:k])
        eplan.solve(fh, uh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eplan.solve(fh, uh)
        torch.cuda.synchronize()
        e2e_s = rk.max(time.perf_counter() - t0)
        e2e = {"value": world * e_units / e2e_s, "unit": "unknowns/s", "h2d_bytes_per_step": fh.numel() * 8,
               "d2h_bytes_per_step": uh.numel() * 8}
        if k < len(probs):
            e2e["sample"] = f"first {k} of {len(probs)} problems ({e_units} unknowns): host-memory budget"
            eplan.close()
        del uh
    except (RuntimeError, ValueError, OSError) as exc:  # host memory
        e2e = {"unavailable": str(exc)[:200]}
    if plan is not None:  # (with its device copies of the fields)
        plan.close()
        plan = None
    if freed:  # the device fields again, for the legs below
        f = fh.cuda() if fh is not None and fh.numel() == units else batch_field(probs)
        u = torch.empty_like(f)
    fh = None
    # the library's default tuning on the same batch, for comparison with the tuned step
    default = None
    if tuning is not None:
        with ftoep.Plan(specs) as dplan:
            dms, _, _ = timed(dplan, f, u, max(1, min(args.steps, 5)), 2, rk, local, clocks=False)
        default = {"ms_per_step": rk.max(dms), "tuned_speedup": rk.max(dms) / ms}
    compare = None
    if not args.no_compare:
        other = "fp64" if precision == "mixed" else "mixed"
        specs2 = [ftoep.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space,
                                    ftoep.FP64 if other == "fp64" else ftoep.MIXED) for p in probs]
        u2 = torch.empty_like(f)
        tuning2 = None if args.no_tune else ftoep.autotune_cached(specs2)[0]
        with ftoep.Plan(specs2, tuning=tuning2) as plan2:
            # two warm-up solves: the first runs directly, the second captures the graph, so
            # the timed solve is a replay like the timed steps of the main leg
            ms2, launches2, _ = timed(plan2, f, u2, 1, 2, rk, local, clocks=False)
            solvers2 = [plan2.solver(i) for i in range(len(probs))]
        ms2 = rk.max(ms2)
        fp64u = u2 if other == "fp64" else u
        mixu = u if other == "fp64" else u2
        # relative error per problem, worst case
        worst = 0.0
        off = 0
        for p in probs:
            n = p.M * p.N
            a, b = mixu[off:off + n], fp64u[off:off + n]
            worst = max(worst, float(torch.linalg.norm(a - b) / torch.linalg.norm(b)))
            off += n
        fl2 = {}
        for p, sv in zip(probs, solvers2):
            for kk, vv in work_model(p, other, sv)[0].items():
                fl2[kk] = fl2.get(kk, 0.0) + vv
        solve_flops = fl2["chain"] + fl2["sine"] + fl2["inverse"]
        compare = {"precision": other, "value": world * units / (ms2 * 1e-3), "ms_per_step": ms2,
                   "gpu_launches": launches2, "tuning": tuning2,
                   "mixed_speedup_vs_fp64": (ms2 / ms) if other == "fp64" else (ms / ms2),
                   "mixed_rel_err_vs_fp64_gpu_worst_problem": worst}
        if other == "fp64":
            compare["fp64_tflops_whole_step"] = solve_flops / (ms2 * 1e-3) / 1e12
            compare["fp64_frac_of_peak_whole_step"] = compare["fp64_tflops_whole_step"] / FP64_PEAK_TFLOPS
        del u2
    del f, u
    torch.cuda.empty_cache()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # oracle on a bounded sample: the first 2048 levels of 8 problems (all their points)
        tot_units, tot_s, th = 0, 0.0, 1
        for p in probs[:8]:
            n0 = min(p.N, 2048)
            v, dt, th = time_oracle(p, n0)
            tot_units += p.M * n0
            tot_s += dt
        cpu = {"value": tot_units / tot_s, "unit": "unknowns/s", "cores": th, "kind": "oracle",
               "sample": f"first min(N,2048) levels of the first 8 problems, {tot_s:.1f} s; O(M N^2) direct marching"}
    singles = None
    if not args.no_singles:
        # config 2 (double) and config 3 (mixed) with the library's choices, and config 2 by the
        # inverse-series solve on request (its time and its prefix error beside the default's)
        singles = [run_single("diffusion", "fp64", 10, 3, rk, local), run_single("wave", "mixed", 5, 3, rk, local),
                   run_single("diffusion", "fp64", 10, 3, rk, local, tuning={"solver": 2})]
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f32+f64", "data": "synthetic",
               "config": {"workload": wname, "nprob": len(probs), "unknowns": units, "precision": precision,
                          "tuning": tuning or "library default", "tuning_from_cache": cached,
                          "solvers": {SOLVER_NAMES[k]: solvers.count(k) for k in sorted(set(solvers))},
                          "l2": f"inputs larger than L2 (f = {units * 8 / 1e9:.1f} GB)"},
               "roofline": roof, "kernel_time_share": shares, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": launches, "default_tuning": default, "compare": compare, "singles": singles}
        print(json.dumps(out))
    rk.close()
    return 0


def run_ours(args):
    import torch
    from paper_1710_11593_gb300 import ftoep, workloads as wl

    rk = Ranks()
    world, rank, local = rk.world, rk.rank, rk.local
    torch.cuda.set_device(local)
    ftoep.load()

    p, wname = workload(args.workload, M=args.M, N=args.N)
    precision = args.precision or ("mixed" if args.workload == "wave" else "fp64")
    prec = ftoep.FP64 if precision == "fp64" else ftoep.MIXED
    spec = ftoep.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec, lam=p.lam)
    f = wl.materialize_torch(p.source, p.kind, p.N, p.M, device="cuda")
    u = torch.empty_like(f)
    tuning = {"scheduler": args.scheduler, "solver": args.solver} if (args.scheduler or args.solver) else None
    plan = ftoep.Plan([spec], tuning=tuning)
    ms, launches, clk = timed(plan, f, u, args.steps, args.warmup, rk, local)
    prof = class_profile(plan, f, u)
    ms = rk.max(ms)
    units = p.M * p.N
    value = rk.value(units, ms)
    tot_ms = sum(x[0] for x in prof.values())
    shares = {k: v[0] / max(1e-9, tot_ms) for k, v in prof.items()}
    solver = plan.solver(0)
    fl, by = work_model(p, precision, solver)
    roof = roofline_of(fl, by, prof, ms, precision)

    # end to end: same solve through the C ABI with pinned HOST buffers (copies inside)
    e2e = {"unavailable": "skipped (--no-e2e)"}
    if not args.no_e2e:
        fh = f.cpu().pin_memory()
        uh = torch.empty_like(fh).pin_memory()
        plan.solve(fh, uh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        esteps = max(1, min(args.steps, 3))
        for _ in range(esteps):
            plan.solve(fh, uh)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / esteps
        e2e_s = rk.max(e2e_s)
        e2e = {"value": world * units / e2e_s, "unit": "unknowns/s", "h2d_bytes_per_step": fh.numel() * 8,
               "d2h_bytes_per_step": uh.numel() * 8}
        del fh, uh
    ex = wl.materialize_torch(p.exact, 0, p.N, p.M, device="cuda") if p.exact else None
    disc = float(torch.max(torch.abs(u - ex)).item()) if ex is not None else None
    del ex
    plan.close()

    compare = None
    if not args.no_compare:
        other = "mixed" if precision == "fp64" else "fp64"
        spec2 = ftoep.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space,
                                  ftoep.MIXED if other == "mixed" else ftoep.FP64, lam=p.lam)
        u2 = torch.empty_like(f)
        with ftoep.Plan([spec2], tuning=tuning) as plan2:
            ms2, _, _ = timed(plan2, f, u2, max(1, min(args.steps, 3)), 2, rk, local, clocks=False)
        fp64u = u if precision == "fp64" else u2
        mixu = u2 if precision == "fp64" else u
        rel = float(torch.linalg.norm(mixu - fp64u) / torch.linalg.norm(fp64u))
        compare = {"precision": other, "value": world * units / (ms2 * 1e-3), "ms_per_step": ms2,
                   "mixed_speedup_vs_fp64": (ms / ms2) if other == "mixed" else (ms2 / ms),
                   "mixed_rel_err_vs_fp64_gpu": rel}
        del u2

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nprefix = min(p.N, 4096 if p.M > 1 else p.N)
        v, dt, th = time_oracle(p, nprefix)
        cpu = {"value": v, "unit": "unknowns/s", "cores": th, "kind": "oracle",
               "sample": f"first {nprefix} of {p.N} time steps, all {p.M} points, {dt:.2f} s; O(M N^2) direct marching"}

    if rank == 0:
        Np = 16
        while Np < p.N:
            Np *= 2
        B, L, Sf = tuning_of(precision, Np)
        out = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f32+f64",
               "data": "synthetic",
               "config": {"workload": wname, "M": p.M, "N": p.N, "gamma": p.gamma, "precision": precision,
                          "l2": f"inputs larger than L2 (f = {f.numel() * 8 / 1e9:.2f} GB)",
                          "block": B, "scheduler": args.scheduler or "library choice",
                          "solver": SOLVER_NAMES[solver]},
               "roofline": roof, "kernel_time_share": shares, "cpu_baseline": cpu, "e2e": e2e,
               "clocks": clk, "gpu_launches": launches, "compare": compare,
               "max_abs_err_vs_exact": disc}
        print(json.dumps(out))
    rk.close()
    return 0


def run_twosided(args):
    """Scheme 1 (two-sided ODE, Example 1, gamma 0.5) by the fast conjugate gradient method:
    one step = one solve to relative residual 1e-12 from a zero guess, f resident in HBM."""
    import torch
    from paper_1710_11593_gb300 import ftoep, workloads as wl
    rk = Ranks()
    torch.cuda.set_device(rk.local)
    ftoep.load()
    N = args.N or 2 ** 20
    g, tol = 0.5, 1e-12
    t, fh, uex = wl.two_sided_example1(N, g)
    f = torch.from_numpy(fh).cuda()
    u = torch.zeros_like(f)
    for _ in range(args.warmup):
        u.zero_()
        ft_u, iters, rel = ftoep.two_sided_cg(f, g, u=u, tol=tol)
    torch.cuda.synchronize()
    rk.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u.zero_()
        _, iters, rel = ftoep.two_sided_cg(f, g, u=u, tol=tol)
    torch.cuda.synchronize()
    sec = rk.max((time.perf_counter() - t0) / args.steps)
    err = float(np.sqrt(np.sum((u.cpu().numpy() - uex) ** 2) / N))
    cpu = None
    if rk.rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as orc
        n0 = 4096
        _, f0, _ = wl.two_sided_example1(n0, g)
        c0 = time.perf_counter()
        orc.two_sided_solve(g, f0)
        dt = time.perf_counter() - c0
        cpu = {"value": (n0 - 1) / dt, "unit": "unknowns/s", "cores": orc.default_threads(), "kind": "oracle",
               "sample": f"dense Gaussian elimination of Scheme 1 at N = {n0} ({dt:.2f} s)"}
    if rk.rank == 0:
        print(json.dumps({"metric": "Scheme 1 unknowns/s (fast CG to 1e-12 relative residual)",
                          "value": rk.world * (N - 1) / sec, "unit": "unknowns/s", "n_gpus": rk.world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": f"two_sided_example1_g0.5_N{N}", "tol": tol},
                          "iterations": iters, "relres": rel, "l2_error_vs_exact": err, "cpu_baseline": cpu}))
    rk.close()
    return 0


def run_advection(args):
    """Schemes 2 and 3 of Sec. 3 by the space-order sweep (ftoep_advection_sweep), double:
    Example 2 (Scheme 2, u = t sin pi x) and Example 3 (Scheme 3, u = t^3 x(1-x)) on M nodes
    and N levels; one step = one sweep of each, f resident in HBM."""
    import torch
    from paper_1710_11593_gb300 import ftoep, workloads as wl
    rk = Ranks()
    torch.cuda.set_device(rk.local)
    ftoep.load()
    # Scheme 3 as printed loses stability on finer grids (h = tau = 1/1024 at gamma 1.5: the
    # oracle's own error grows to 2.4e-2), so the default stays at M = 512 nodes
    M, N = args.M or 512, args.N or 16384
    h = 1.0 / M
    g2, g3 = 0.5, 1.5
    xm = (np.arange(1, M + 1) - 0.5) * h
    x = np.arange(1, M + 1) * h
    t, th = wl.time_points(0, N), wl.time_points(1, N)
    f2 = np.outer(np.sin(np.pi * xm), t ** (1 - g2) / math.gamma(2 - g2)) + np.outer(np.pi * np.cos(np.pi * xm), t)
    f3 = np.outer(x - x * x, 6 * th ** (3 - g3) / math.gamma(4 - g3)) + np.outer(1 - 2 * x, th ** 3)
    d2, d3 = torch.from_numpy(f2).cuda(), torch.from_numpy(f3).cuda()
    u2, u3 = torch.empty_like(d2), torch.empty_like(d3)
    for _ in range(args.warmup):
        ftoep.advection_sweep(2, d2, g2, u=u2)
        ftoep.advection_sweep(3, d3, g3, u=u3)
    torch.cuda.synchronize()
    rk.barrier()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    for _ in range(args.steps):
        ftoep.advection_sweep(2, d2, g2, u=u2)
    e1.record()
    for _ in range(args.steps):
        ftoep.advection_sweep(3, d3, g3, u=u3)
    e2.record()
    torch.cuda.synchronize()
    ms2, ms3 = rk.max(e0.elapsed_time(e1) / args.steps), rk.max(e1.elapsed_time(e2) / args.steps)
    err2 = float(np.sqrt(h * np.sum((u2[:-1, -1].cpu().numpy() - np.sin(np.pi * x[:-1])) ** 2)))
    err3 = float(np.sqrt(h * np.sum((u3[:-1, -1].cpu().numpy() - (x - x * x)[:-1]) ** 2)))
    cpu = None
    if rk.rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as orc
        n0 = 512  # the oracle's direct method on the first n0 levels (O(M n0^2))
        c0 = time.perf_counter()
        ref = orc.advection_march(2, g2, f2[:, :n0], T=n0 / N)
        dt = time.perf_counter() - c0
        rel = float(np.max(np.abs(u2[:, :n0].cpu().numpy() - ref)) / np.max(np.abs(ref)))
        cpu = {"value": M * n0 / dt, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
               "sample": f"direct method of Scheme 2 on the first {n0} levels, all {M} nodes ({dt:.2f} s)",
               "gpu_rel_err_on_sample": rel}
    if rk.rank == 0:
        print(json.dumps({"metric": "advection sweep unknowns/s (Scheme 2, Example 2; Scheme 3 beside)",
                          "value": rk.world * M * N / (ms2 * 1e-3), "unit": "unknowns/s", "n_gpus": rk.world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms2, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": f"advection_example2_g{g2}_M{M}_N{N}"},
                          "l2_error_vs_exact": err2,
                          "scheme3": {"workload": f"advection_example3_g{g3}_M{M}_N{N}", "ms_per_step": ms3,
                                      "value": M * N / (ms3 * 1e-3), "l2_error_vs_exact": err3},
                          "cpu_baseline": cpu}))
    rk.close()
    return 0


def run_adjoint(args):
    """Config 5 (gamma 0.6, M 1023, N 65536, double): one step = the forward solve and the
    adjoint (dL/df and dL/dgamma) of L = ||u(., T) - u_obs||^2, f resident in HBM; the gradient
    in gamma checked against central differences of the GPU forward solve."""
    import torch
    from paper_1710_11593_gb300 import ftoep, workloads as wl
    rk = Ranks()
    torch.cuda.set_device(rk.local)
    ftoep.load()
    M, N, g = args.M or 1023, args.N or 65536, 0.6
    p = wl.config_adjoint(M=M, N=N, gamma=g)
    f = wl.materialize_torch(p.source, p.kind, N, M, device="cuda")
    spec = ftoep.ProblemSpec(p.kind, g, N, M, p.space, ftoep.FP64)
    with ftoep.Plan([ftoep.ProblemSpec(p.kind, 0.55, N, M, p.space, ftoep.FP64)]) as p55:
        u_obs = p55.solve(f)[:, -1].clone() + torch.from_numpy(wl.noise(M, 1e-3, seed=2)).cuda()
    with ftoep.Plan([spec]) as plan:
        u = plan.solve(f)
        gg = torch.zeros_like(u)

        def step():
            plan.solve(f, u)
            gg[:, -1] = 2.0 * (u[:, -1] - u_obs)
            return plan.adjoint(gg, u)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            dldf, dg = step()
        e1.record()
        torch.cuda.synchronize()
        ms = rk.max(e0.elapsed_time(e1) / args.steps)
        dg = float(dg[0])
    fd = None
    hstep = 1e-6
    vals = []
    for gm in (g - hstep, g + hstep):
        with ftoep.Plan([ftoep.ProblemSpec(p.kind, gm, N, M, p.space, ftoep.FP64)]) as pp:
            uu = pp.solve(f)
            vals.append(float(torch.sum((uu[:, -1] - u_obs) ** 2)))
    fd = (vals[1] - vals[0]) / (2 * hstep)
    if rk.rank == 0:
        print(json.dumps({"metric": "forward + adjoint unknowns/s (config 5, double)",
                          "value": rk.world * M * N / (ms * 1e-3), "unit": "unknowns/s", "n_gpus": rk.world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": f"adjoint_g{g}_M{M}_N{N}"},
                          "dldgamma": dg, "dldgamma_central_difference": fd,
                          "rel_diff_vs_central_difference": abs(dg - fd) / abs(fd)}))
    rk.close()
    return 0


def run_gmres(args):
    """Restarted GMRES(40) of Sec. 3.2 against the direct solve on the config-2 family (double,
    sub-diffusion): one step = one GMRES solve to relative residual 1e-12 from zero."""
    import torch
    from paper_1710_11593_gb300 import ftoep, workloads as wl
    rk = Ranks()
    torch.cuda.set_device(rk.local)
    ftoep.load()
    p = wl.config_diffusion(M=args.M or 255, N=args.N or 16384)
    f = wl.materialize_torch(p.source, p.kind, p.N, p.M, device="cuda")
    with ftoep.Plan([ftoep.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, ftoep.FP64)]) as plan:
        ud = plan.solve(f)
        for _ in range(args.warmup):
            u, it, rr = plan.gmres(f, restart=40, tol=1e-12, maxit=100000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            u, it, rr = plan.gmres(f, restart=40, tol=1e-12, maxit=100000)
        torch.cuda.synchronize()
        sec = rk.max((time.perf_counter() - t0) / args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            plan.solve(f, ud)
        e1.record()
        torch.cuda.synchronize()
        direct_ms = e0.elapsed_time(e1) / args.steps
    rel = float(torch.linalg.norm(u - ud) / torch.linalg.norm(ud))
    if rk.rank == 0:
        print(json.dumps({"metric": "GMRES(40) unknowns/s on the config-2 family (direct solve beside)",
                          "value": rk.world * p.M * p.N / sec, "unit": "unknowns/s", "n_gpus": rk.world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": f"gmres_diffusion_g{p.gamma}_M{p.M}_N{p.N}",
                                                          "restart": 40, "tol": 1e-12},
                          "iterations": it, "relres": rr, "rel_diff_vs_direct_solve": rel,
                          "direct_solve_ms": direct_ms}))
    rk.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "twosided":
        return run_twosided(args)
    if args.workload == "advection":
        return run_advection(args)
    if args.workload == "gmres":
        return run_gmres(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
