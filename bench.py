#!/usr/bin/env python3
"""Benchmark: fine-grid unknowns/s of one FMG-FAS-SR solve on GB300.

Workload (default): -u'' = f on (0,1), u(0) = u(1) = 0, N = 2^24 cells,
4096 SR segments of 4096 cells with 8 buffer cells, one FMG cycle of
V(1,1) FAS cycles, lexicographic Gauss-Seidel, FP64; f from the exact
solution u = sum_{k=1..32} c_k sin(k pi x), c_k ~ N(0,1)/k^2 (seed 1).

One step = one srfmg_solve (the whole hot path: rhs hierarchy, FMG steps,
fused SR pre- and post-leg).  Inputs are resident in HBM; the timed region is
bracketed by a barrier and a device synchronisation and timed with CUDA events
on the launching stream; f, u and the workspace (about 640 MiB) exceed the
129 MB L2, so no flush is needed between steps.  The JSON line also carries:
e2e (a stream of srfmg_solve_host_async calls from pinned host buffers: every
step copies its f in and its u out, overlapping the neighbouring steps'
solves; e2e.serial: srfmg_solve_host, one synchronous step at a time), the
plain FP64 stored-grid FMG-FAS on the same GPU, the roofline of
the dominant kernel, the oracle on the host cores, clocks sampled during the
timed region, and the accuracy of the result against the exact solution.

The default line also carries the other workloads under their own keys
(each with its plain FP64 stored-grid baseline and accuracy flags): "batch"
(the batch of variable-coefficient problems below, mixed precision) and
"bratu" (the Bratu problem at N = 2^26, mixed precision); "plain_fixed" (plain
stored FMG-FAS in the same fixed point, which separates what segmental
refinement adds from what the arithmetic adds); "alu_peak" (measured
integer, FP64 and FP32 throughput, srfmg_alu_peaks) and
"cpu_baseline_allcores" (the oracle on every host core, one independent solve
per core).  --quick leaves those out.

--impl reference times the CPU oracle (the method's plain serial C
restatement) on the host cores: one solve of the full workload per step
(a bounded sample for Bratu and the batch, stated in its config).

--workload batch: 8192 independent problems of N = 2^m cells, m ~ U{10..20}
(seed 11; about 1.55e9 unknowns in all), each -(a u')' = f with its own
seeded a = exp(g/2) (16 cosine modes) and 32-mode sine solution (--batch-op
laplace: -u'' = f, 64-bit fixed point); one srfmg group: a batched plan per
size with its segment layout autotuned (--no-tune: min(4096, N/4)-cell
segments, 8 buffer cells), all replayed as one CUDA graph with a branch per
size; mixed precision.  value = all problems' unknowns / time of one group
solve.

--workload varcoef: -(a u')' = f, a = exp(g/2) at the faces with g a seeded
16-mode cosine series, N = 2^24 cells, 4096 segments of 4096 cells, V(1,1);
u = sum_{k=1..16} c_k sin(k pi x) (seed 1).

--workload bratu: the nonlinear -u'' + lam e^u = f (lam = 1) with the same
discretisation and FAS cycles, N = 2^26 cells, 16384 segments of 4096 cells,
V(2,1); u = 1/2 sum_{k=1..16} c_k sin(k pi x) (seed 1).

--precision mixed (default): 64-bit fixed point for -u'' = f; for the
variable coefficient and Bratu, FP64 residuals, tau, interpolations and
coarsest solves with FP32 Gauss-Seidel correction recurrences.

Multi-GPU: the solve does not shard across GPUs here; with --gpus N every rank
solves its own copy (replicas, weak scaling) and the value is the sum over
ranks with the time taken as the maximum over ranks.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine-grid unknowns/s per FMG-FAS-SR solve at discretization accuracy vs plain FP64"
METRIC_BATCH = ("fine-grid unknowns/s over a batch of independent FMG-FAS-SR solves at "
                "discretization accuracy vs plain FP64")
METRIC_VARCOEF = ("fine-grid unknowns/s per FMG-FAS-SR solve of -(a u')'=f at discretization accuracy "
                  "vs plain FP64")
METRIC_BRATU = ("fine-grid unknowns/s per FMG-FAS-SR solve of -u''+lam e^u=f at discretization "
                "accuracy vs plain FP64")
UNIT = "unknowns/s"
NOMINAL_FP64_TFLOPS = 1.26        # 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")

# Algorithmic FP64 flops per cell of each launch kind (residual-form method
# arithmetic, sequential sweep; exact power-of-two scalings not counted) and
# algorithmic DRAM bytes per cell of the level the launch sweeps.
FLOPS_PER_CELL = {"sr_post": 13.5, "sr_pre": 15.5, "level_down_fmg": 15.5,
                  "level_down": 9.0, "level_up": 9.0}
# Bratu, V(2,1): the nonlinear sweep adds 4 per cell (c e^u with the
# exponential counted as one operation, the diagonal 2 + e, its reciprocal,
# the residual term) and tau 5 (three exponentials, two combinations)
# variable coefficient, V(1,1): every flux and diagonal weighted (sweep 5 + 3:
# two products and the reciprocal of the diagonal; tau 3 more)
FLOPS_PER_CELL_VARCOEF = {"sr_post": 6.5 + 1 * (2 + 8), "sr_pre": 6.5 + 8 + 0.5 + 6.5,
                          "level_down_fmg": 6.5 + 8 + 0.5 + 6.5, "level_down": 8 + 0.5 + 6.5,
                          "level_up": 2.0 + 8}
FLOPS_PER_CELL_BRATU = {"sr_post": 6.5 + 1 * (2 + 9), "sr_pre": 6.5 + 2 * 9 + 0.5 + 6,
                        "level_down_fmg": 6.5 + 2 * 9 + 0.5 + 6, "level_down": 2 * 9 + 0.5 + 6,
                        "level_up": 2.0 + 1 * 9}
# mixed precision of the Bratu problem: the Newton Gauss-Seidel recurrence, the Newton
# denominator and its reciprocal run in FP32; the FP64 part of a sweep is the residual
# (flux, flux difference, residual, c e^u and its term) and the update
FLOPS_PER_CELL_BRATU_MX = {"sr_post": 6.5 + 1 * (2 + 6), "sr_pre": 6.5 + 2 * 6 + 0.5 + 6,
                           "level_down_fmg": 6.5 + 2 * 6 + 0.5 + 6, "level_down": 2 * 6 + 0.5 + 6,
                           "level_up": 2.0 + 1 * 6}
# the fixed-point variable coefficient also reads its face words A (8 B per face)
# and two multiplier words per cell (16 B) in every sweeping kernel
BYTES_PER_CELL_VC_FX = {"sr_post": 44.0, "sr_pre": 44.0, "level_down_fmg": 44.0, "level_down": 48.0,
                        "level_up": 52.0}
STREAMING = ("sr_pre", "sr_post", "level_down_fmg", "level_down", "level_up")
BYTES_PER_CELL = {"sr_post": 20.0, "sr_pre": 20.0, "level_down_fmg": 20.0,
                  "level_down": 24.0, "level_up": 28.0, "rhs_hierarchy": 16.0}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["srfmg", "reference"], default="srfmg")
    ap.add_argument("--workload", choices=["poisson", "bratu", "varcoef", "batch"], default="poisson")
    ap.add_argument("--nprob", type=int, default=None, help="batch: number of problems (8192; 1024 for bratu)")
    ap.add_argument("--lam", type=float, default=1.0, help="Bratu: lam of -u'' + lam e^u = f")
    ap.add_argument("--log2n", type=int, default=None, help="default 24 (poisson), 26 (bratu)")
    ap.add_argument("--segment-width", type=int, default=4096)
    ap.add_argument("--buffer-width", type=int, default=8)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed",
                    help="mixed: 64-bit fixed point for solution/residual/tau, FP64 coarse solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch: fixed segment layout min(4096, N/4), buffer 8, instead of autotuning each size")
    ap.add_argument("--batch-op", choices=["varcoef", "laplace", "bratu"], default="varcoef",
                    help="batch: operator of the problems (bratu: 1024 problems, m ~ U{12..18}, V(2,1))")
    ap.add_argument("--quick", action="store_true",
                    help="leave the batch, Bratu, all-core oracle and ALU probes out of the default line")
    ap.add_argument("--shape", default=None,
                    help="TAIL,TILE,CHAIN_DOWN,CHAIN_UP: the headline plan's CTA shape instead of the shape "
                         "autotuner's choice (every shape gives the same bits; for profiling runs)")
    ap.add_argument("--only-solve", action="store_true",
                    help="time the SR solve only (no plain baseline, e2e, profile or CPU leg); "
                         "the minimal run used for ncu captures")
    a = ap.parse_args()
    if a.log2n is None:
        a.log2n = 26 if a.workload == "bratu" else 24
    if a.nprob is None:
        a.nprob = 1024 if a.batch_op == "bratu" else 8192
    return a


def precision_text(op, precision):
    if precision == "fp64":
        return "FP64"
    if op == "laplace":
        return "64-bit fixed point (solution, residual, tau, interpolation) + FP64 coarsest solve"
    if op == "varcoef":
        return ("64-bit fixed point (solution, residual with exact 128-bit fluxes, tau, interpolation; 63-bit "
                "Gauss-Seidel multipliers) + FP64 coarsest solve")
    return ("mixed: FP64 solution, residual, tau, interpolation and coarsest solve (e^u of the residual and tau "
            "by a table-driven FP64 exponential, < 1.5e-13 relative); FP32 Gauss-Seidel corrections")


def workload_config(a):
    if getattr(a, "workload", "poisson") == "varcoef":
        return {
            "workload": f"1D -(a u')'=f, a=exp(g/2) (8-mode cosine series g, seed 1), N=2^{a.log2n}, FMG-FAS "
                        f"V(1,1) lexicographic GS, 1 SR level of {(1 << a.log2n) // a.segment_width} segments x "
                        f"{a.segment_width} cells, buffer {a.buffer_width}, {precision_text('varcoef', a.precision)}",
            "precision": a.precision, "N": 1 << a.log2n, "segment_width": a.segment_width,
            "buffer_width": a.buffer_width, "n_sr_levels": 1, "nu": [1, 1], "coarsest_level": 2,
            "modes": 16, "seed": 1,
            "l2": "inputs larger than L2 (f and u 128 MiB each, log a 128 MiB, the stored levels)",
        }
    if getattr(a, "workload", "poisson") == "batch" and getattr(a, "batch_op", "varcoef") == "bratu":
        return {
            "workload": f"{a.nprob} independent 1D -u''+lam e^u=f problems (lam={a.lam}), N=2^m with m ~ "
                        f"U{{12..18}} (seed 11), FMG-FAS V(2,1) pointwise Newton lexicographic GS, 1 SR level, "
                        f"buffer 8, {precision_text('bratu', 'mixed')}; one srfmg group",
            "operator": "bratu", "lam": a.lam, "precision": "mixed", "nprob": a.nprob, "m_range": [12, 18],
            "size_seed": 11, "modes": 16, "buffer_width": 8, "n_sr_levels": 1, "nu": [2, 1],
            "coarsest_level": 2, "l2": "inputs larger than L2 (about 0.6 GB of f and of u)",
        }
    if getattr(a, "workload", "poisson") == "batch":
        op = getattr(a, "batch_op", "varcoef")
        eq = "-(a u')'=f, a=exp(g/2) (16-mode cosine series g per problem)" if op == "varcoef" else "-u''=f"
        return {
            "workload": f"{a.nprob} independent 1D {eq} problems, N=2^m with m ~ U{{10..20}} (seed 11), "
                        f"FMG-FAS V(1,1) lexicographic GS, 1 SR level, buffer 8, "
                        f"{precision_text(op, 'mixed')}; one srfmg group (a batched plan per size, all sizes "
                        f"replayed as one CUDA graph with a branch per size)",
            "operator": op, "precision": "mixed", "nprob": a.nprob, "m_range": [10, 20], "size_seed": 11,
            "modes": 32, "buffer_width": 8, "n_sr_levels": 1, "nu": [1, 1], "coarsest_level": 2,
            "l2": "inputs larger than L2 (about 12 GB of f and 12 GB of u)",
        }
    if getattr(a, "workload", "poisson") == "bratu":
        return {
            "workload": f"1D -u''+lam e^u=f, lam={a.lam}, N=2^{a.log2n}, FMG-FAS V(2,1) pointwise Newton "
                        f"lexicographic GS, 1 SR level of {(1 << a.log2n) // a.segment_width} segments x "
                        f"{a.segment_width} cells, buffer {a.buffer_width}, {precision_text('bratu', a.precision)}",
            "precision": a.precision, "N": 1 << a.log2n, "segment_width": a.segment_width,
            "buffer_width": a.buffer_width, "n_sr_levels": 1, "nu": [2, 1], "coarsest_level": 2,
            "lam": a.lam, "modes": 16, "seed": 1,
            "l2": "inputs larger than L2 (f and u 512 MiB each plus the stored coarse levels)",
        }
    prec = ("64-bit fixed point (solution, residual, tau, interpolation) + FP64 coarsest solve"
            if getattr(a, "precision", "fp64") == "mixed" else "FP64")
    return {
        "workload": f"1D -u''=f, N=2^{a.log2n}, FMG-FAS V(1,1) lexicographic GS, 1 SR level of "
                    f"{(1 << a.log2n) // a.segment_width} segments x {a.segment_width} cells, "
                    f"buffer {a.buffer_width}, {prec}",
        "precision": getattr(a, "precision", "fp64"),
        "N": 1 << a.log2n, "segment_width": a.segment_width, "buffer_width": a.buffer_width,
        "n_sr_levels": 1, "nu": [1, 1], "coarsest_level": 2, "modes": 32, "seed": 1,
        "l2": "inputs larger than L2 (f and u 128 MiB each plus the stored coarse levels)",
    }


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, want_gpus, use_cuda):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if use_cuda else "gloo"
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64,
                         device="cuda" if self.pg.get_backend() == "nccl" else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="srfmg_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def kernel_source_hash():
    h = hashlib.sha256()
    for rel in ("paper_1207_6720_gb300/csrc/srfmg_kernels.cuh", "paper_1207_6720_gb300/csrc/srfmg_fixed.cuh",
                "paper_1207_6720_gb300/csrc/srfmg.cu"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_field(kernel_kind, precision, field):
    """A per-launch figure (`field`: dram_bytes_per_full_launch or
    warp_inst_per_full_launch) of `kernel_kind` from the committed ncu summary,
    or None if there is none or the kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel_kind}_{precision}_ncu.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_src = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m_b = re.search(field + r":\s*([0-9.eE+]+)", text)
    if not (m_src and m_b) or m_src.group(1) != kernel_source_hash():
        return None
    return float(m_b.group(1))


def recorded_traffic(kernel_kind, precision):
    return recorded_field(kernel_kind, precision, "dram_bytes_per_full_launch")


_ALU = None


def alu_peak(dev):
    """Measured integer, FP64 and FP32 throughput of the device (srfmg_alu_peaks),
    once per process."""
    global _ALU
    if _ALU is None:
        from paper_1207_6720_gb300 import srfmg
        _ALU = srfmg.alu_peaks(dev)
    return _ALU


def fp64_peak_tflops():
    if _ALU:
        return _ALU["fp64_flops"] / 1e12, "measured FP64 FMA throughput (srfmg_alu_peaks)"
    return NOMINAL_FP64_TFLOPS, "nominal FP64 from unit counts and the maximum SM clock"


def measured_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def cpu_baseline(f, M, W, b, u_exact):
    """The CPU oracle (serial C, FP64) on the full workload, repeated for
    about 10 s; also returns the oracle's error against the exact solution."""
    import oracle
    p = oracle.sr_params(M, W, b, nRS=1)
    t0 = time.perf_counter()
    ref = oracle.fmg_v(p, f)
    reps, elapsed = 1, time.perf_counter() - t0
    while elapsed < 10.0 and reps < 20:
        oracle.fmg_v(p, f)
        reps += 1
        elapsed = time.perf_counter() - t0
    value = reps * (1 << M) / elapsed
    return ref, {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                 "sample": f"{reps} serial solves of the full N=2^{M} workload "
                           f"(C oracle, serial SR with the finest level never stored)"}


_AC_F = None


def _allcore_init(M):
    global _AC_F
    import oracle
    from paper_1207_6720_gb300 import workloads
    oracle.lib()
    _AC_F = workloads.sine_series(M, 32, seed=1)[0]


def _allcore_solve(args):
    import oracle
    M, W, b = args
    oracle.fmg_v(oracle.sr_params(M, W, b, nRS=1), _AC_F)
    return 1


def cpu_baseline_allcores(M, W, b):
    """The oracle as it stands on every host core at once: one independent
    serial solve of the full workload per core (processes started with spawn),
    after one untimed round; value = cores x N / wall time of the round."""
    import multiprocessing as mp
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(n, initializer=_allcore_init, initargs=(M,)) as pool:
        pool.map(_allcore_solve, [(M, W, b)] * n, chunksize=1)
        t0 = time.perf_counter()
        pool.map(_allcore_solve, [(M, W, b)] * n, chunksize=1)
        dt = time.perf_counter() - t0
    return {"value": n * (1 << M) / dt, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} concurrent serial solves of the full N=2^{M} workload, one per host core "
                      f"(C oracle, serial SR), wall time of one round"}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(a):
    dist = Dist(a.gpus, use_cuda=False)
    if dist.rank != 0:
        dist.close()
        return
    import oracle
    from paper_1207_6720_gb300 import workloads
    # one solve per step: the full workload for the Poisson and variable-coefficient
    # problems (about 2 s per solve at N = 2^24 on one core) when warm-up and timed
    # steps fit about 150 s of oracle time, else a bounded sample of the largest size
    # that does (the rate of one untimed solve at N = 2^18 sets it); at most N = 2^22
    # for the Bratu problem (its N = 2^26 solve takes about 12 s) and one problem of
    # the batch's largest size for the batch
    Mmax = {"bratu": min(a.log2n, 22), "batch": 20}.get(a.workload, a.log2n)

    def problem(Ms):
        Ws = min(a.segment_width, (1 << Ms) // 4)
        if a.workload == "bratu":
            f, _, _ = workloads.bratu_series(Ms, 16, seed=1, lam=a.lam)
            return f, oracle.sr_params(Ms, Ws, a.buffer_width, nRS=1, nu1=2, nu2=1, op="bratu", lam=a.lam)
        if a.workload == "varcoef":
            f, _, log_a = workloads.varcoef_series(Ms, 16, seed=1)
            return f, oracle.sr_params(Ms, Ws, a.buffer_width, nRS=1, op="varcoef", coef=np.exp(log_a))
        f, _, _ = workloads.sine_series(Ms, 32, seed=1)
        return f, oracle.sr_params(Ms, Ws, a.buffer_width, nRS=1)

    Mcal = min(Mmax, 18)
    f, p = problem(Mcal)
    t0 = time.perf_counter()
    oracle.fmg_v(p, f)
    rate = (1 << Mcal) / (time.perf_counter() - t0)
    Ms = Mmax
    while Ms > 16 and (a.warmup + a.steps) * (1 << Ms) / rate > 150.0:
        Ms -= 1
    f, p = problem(Ms)
    for _ in range(a.warmup):
        oracle.fmg_v(p, f)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.fmg_v(p, f)
    dt = time.perf_counter() - t0
    value = a.steps * (1 << Ms) / dt
    sample = f"one serial oracle solve of the workload at N=2^{Ms} per step"
    if a.workload == "batch":
        sample = f"one serial oracle solve of a problem of the batch's family at N=2^{Ms} per step"
    config = workload_config(a)
    if a.workload != "batch" and Ms != a.log2n:
        config = dict(config, N=1 << Ms, sampled=f"N=2^{Ms} solved per step instead of the workload's "
                                                 f"2^{a.log2n} (a bounded sample)")
    line = {"metric": {"bratu": METRIC_BRATU, "varcoef": METRIC_VARCOEF, "batch": METRIC_BATCH}.get(a.workload, METRIC),
            "value": value, "unit": UNIT,
            "impl": "reference",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    dist.close()


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def tuned_solver(srfmg, M, dev, reps=3, coef=None, shape=None, **kw):
    """A plan with its CTA shape (coarse tail extent, cells per tile of the stored
    levels of at most 2^18 cells, chained passes) picked by srfmg_autotune_shape
    before any timing, or `shape` (TAIL,TILE,CHAIN_DOWN,CHAIN_UP) when given; the
    shape changes no bit of the result.  coef: log a for the variable
    coefficient (the tuning solves use a = 1)."""
    if shape:
        t, c, cd, cu = (int(x) for x in shape.split(","))
        best = srfmg.default_params(M, tail_level=t, tile_cells=c, chain_down=cd, chain_up=cu, **kw)
        s = srfmg.Solver(M, device=dev, params=best)
        if coef is not None:
            s.set_coefficient(coef)
        return s, {"tail_level": t, "tile_cells": c, "chain_down": cd, "chain_up": cu, "given": True}
    best, table = srfmg.autotune_shape(srfmg.default_params(M, **kw), device=dev, reps=reps)
    s = srfmg.Solver(M, device=dev, params=best)
    if coef is not None:
        s.set_coefficient(coef)
    shape = {"tail_level": best.tail_level, "tile_cells": best.tile_cells,
             "chain_down": best.chain_down, "chain_up": best.chain_up,
             "candidates_ms": {f"T{t}_C{c}" + (f"_D{cd}_U{cu}" if cd or cu else ""): round(ms, 4)
                               for t, c, cd, cu, ms in table}}
    return s, shape


def time_solves(solver, fd, ud, steps, warmup, dist, stream):
    import torch
    for _ in range(warmup):
        solver.solve(fd, ud, stream=stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        solver.solve(fd, ud, stream=stream)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    dist.barrier()
    return e0.elapsed_time(e1) / steps


def run_gpu(a):
    import torch
    from paper_1207_6720_gb300 import srfmg, workloads

    dist = Dist(a.gpus, use_cuda=True)
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    M, W, b = a.log2n, a.segment_width, a.buffer_width
    N = 1 << M
    f, u_exact, _ = workloads.sine_series(M, 32, seed=1)
    fd = torch.from_numpy(f).to(dev)
    ud = torch.empty_like(fd)

    prec = srfmg.MIXED if a.precision == "mixed" else srfmg.FP64
    solver, shape = tuned_solver(srfmg, M, dev, shape=a.shape, segment_width=W, buffer_width=b, precision=prec)
    info = solver.info()

    sampler = ClockSampler(dev)
    sampler.start()
    ms = time_solves(solver, fd, ud, a.steps, a.warmup, dist, stream)
    clocks = sampler.stop()
    ms = dist.max(ms)
    value = dist.world * N / (ms * 1e-3)
    u = ud.cpu().numpy()
    if a.only_solve:
        if dist.rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms,
                              "steps": a.steps, "warmup": a.warmup, "config": workload_config(a),
                              "gpu_launches": info.kernels_per_solve * a.steps}), flush=True)
        solver.close()
        dist.close()
        return

    # plain FP64 stored-grid FMG-FAS (every level stored, no SR) on the same GPU
    plain, _ = tuned_solver(srfmg, M, dev, n_sr_levels=0)
    ms_plain = dist.max(time_solves(plain, fd, ud, max(10, a.steps // 4), a.warmup, dist, stream))
    u_plain = ud.cpu().numpy()
    plain_info = plain.info()
    plain.close()
    # plain stored-grid FMG-FAS in the same arithmetic as the headline: what SR itself
    # adds or costs on this GPU, apart from the arithmetic
    plain_fixed = None
    if prec != srfmg.FP64:
        pfx, _ = tuned_solver(srfmg, M, dev, n_sr_levels=0, precision=prec)
        ms_pfx = dist.max(time_solves(pfx, fd, ud, max(10, a.steps // 4), a.warmup, dist, stream))
        u_pfx = ud.cpu().numpy()
        plain_fixed = {"value": dist.world * N / (ms_pfx * 1e-3), "ms_per_step": ms_pfx,
                       "kernels_per_solve": pfx.info().kernels_per_solve, "sr_speedup_over_it": ms_pfx / ms,
                       "err_max_vs_exact": float(np.max(np.abs(u_pfx - u_exact)))}
        pfx.close()
    # the same SR solve in FP64 arithmetic (when the headline is the fixed-point one)
    sr64 = None
    if prec != srfmg.FP64:
        s64 = srfmg.Solver(M, device=dev, segment_width=W, buffer_width=b, precision=srfmg.FP64)
        ms64 = dist.max(time_solves(s64, fd, ud, max(10, a.steps // 4), a.warmup, dist, stream))
        u64 = ud.cpu().numpy()
        s64.close()
        sr64 = {"value": dist.world * N / (ms64 * 1e-3), "ms_per_step": ms64,
                "err_max_vs_exact": float(np.max(np.abs(u64 - u_exact)))}

    # two SR levels (levels M and M-1 segmented; Fig. 3 with a deeper SR set)
    s2 = srfmg.Solver(M, device=dev, n_sr_levels=2, segment_width=W, buffer_width=b, precision=prec)
    ms2 = dist.max(time_solves(s2, fd, ud, max(10, a.steps // 4), a.warmup, dist, stream))
    u2 = ud.cpu().numpy()
    s2.close()
    sr2 = {"value": dist.world * N / (ms2 * 1e-3), "ms_per_step": ms2,
           "err_max_vs_exact": float(np.max(np.abs(u2 - u_exact)))}

    # autotuner (row f1): the fastest admissible segment layout for this solve
    best, table = srfmg.autotune(M, device=dev, reps=5, precision=prec)
    autotune = {"choice": {"segment_width": best.segment_width, "buffer_width": best.buffer_width},
                "candidates_ms": {f"W{w}_b{bb}": round(t, 4) for w, bb, t in table},
                "benchmarked_layout": {"segment_width": W, "buffer_width": b}}

    # adjoint solve (dL/df for L = 1/2 |u - u_obs|^2, u_obs = exact + N(0, 1e-3^2))
    rng = np.random.default_rng(7)
    g_adj = torch.from_numpy(u - (u_exact + rng.normal(0.0, 1e-3, N))).to(dev)
    lam = torch.empty_like(g_adj)

    class _Adj:
        def solve(self, x, y, stream=None):
            return solver.adjoint(x, y, stream=stream)
    ms_adj = dist.max(time_solves(_Adj(), g_adj, lam, max(10, a.steps // 4), a.warmup, dist, stream))
    adjoint = {"value": dist.world * N / (ms_adj * 1e-3), "unit": UNIT, "ms_per_step": ms_adj,
               "rhs": "u - u_obs, u_obs = exact + N(0, 1e-3^2), seed 7"}

    # functionals only (Fig. 3, the paper's section on obtaining the solution): the
    # same SR solve with the fine grid never written, the functionals of the fine
    # solution reduced on the fly; timed without and with a reference (the exact
    # solution, which adds its 128 MiB read and the error functionals)
    ue_d = torch.from_numpy(u_exact).to(dev)
    fo = torch.empty(srfmg.NUM_FUNCTIONALS, dtype=torch.float64, device=dev)

    class _Fn:
        def __init__(self, ref):
            self.ref = ref

        def solve(self, x, y, stream=None):
            return solver.solve_functionals(x, None, self.ref, out=fo, stream=stream)
    fn_steps = max(10, a.steps // 4)
    ms_fn = dist.max(time_solves(_Fn(None), fd, ud, fn_steps, a.warmup, dist, stream))
    ms_fn_ref = dist.max(time_solves(_Fn(ue_d), fd, ud, fn_steps, a.warmup, dist, stream))
    fvals = fo.cpu().numpy()
    functionals = {"value": dist.world * N / (ms_fn * 1e-3), "unit": UNIT, "ms_per_step": ms_fn,
                   "ms_per_step_with_reference": ms_fn_ref, "fine_grid_written": False,
                   "functionals": {"h_sum_u": float(fvals[0]), "h_sum_u2": float(fvals[1]),
                                   "max_abs_u": float(fvals[2]), "h_sum_err2_vs_exact": float(fvals[3]),
                                   "max_abs_err_vs_exact": float(fvals[4])}}
    del ue_d

    # end to end through the public API from pinned host buffers
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.empty(N, dtype=torch.float64).pin_memory()
    fh_np, uh_np = fh.numpy(), uh.numpy()
    for _ in range(2):
        solver.solve_host(fh_np, uh_np, stream=stream)
    dist.barrier()
    e2e_steps = max(5, a.steps // 10)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.solve_host(fh_np, uh_np, stream=stream)
    dt_serial = dist.max((time.perf_counter() - t0) / e2e_steps)
    # a stream of solves from host memory (srfmg_solve_host_async): every step copies its f
    # in and its u out, overlapping the neighbouring steps' solves
    for _ in range(3):
        solver.solve_host_async(fh_np, uh_np, stream=stream)
    solver.host_join(stream=stream)
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.solve_host_async(fh_np, uh_np, stream=stream)
    solver.host_join(stream=stream)
    torch.cuda.synchronize()
    dt_e2e = dist.max((time.perf_counter() - t0) / e2e_steps)
    e2e = {"value": dist.world * N / dt_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(f.nbytes), "d2h_bytes_per_step": int(uh_np.nbytes),
           "mode": f"srfmg_solve_host_async: {e2e_steps} pipelined solves from pinned host buffers, each "
                   f"copying its f in and its u out, timed on the host clock from the first call to the join",
           "serial": {"value": dist.world * N / dt_serial, "unit": UNIT,
                      "mode": "srfmg_solve_host: copy in, solve, copy out, synchronise, one step at a time"}}

    # per-launch durations (CUDA events around every kernel on this stream)
    prof = solver.profile(fd, torch.empty_like(fd), nsolves=5, stream=stream)
    torch.cuda.synchronize()
    top_name, top_ms = max(prof, key=lambda x: x[1])
    kind, lvl = top_name.split(" L")
    kind = kind.replace("fx.", "")
    cells = 1 << int(lvl)
    peaks = measured_peaks()
    flops = FLOPS_PER_CELL.get(kind, 0.0) * cells
    achieved_tf = flops / (top_ms * 1e-3) / 1e12
    bytes_alg = BYTES_PER_CELL.get(kind, 0.0) * cells
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    traffic = recorded_traffic(kind, a.precision)
    alu = alu_peak(dev)
    fp64_peak, fp64_src = fp64_peak_tflops()
    hbm_achieved = bytes_alg / (top_ms * 1e-3) / 1e9
    hbm_view = {"bound": "hbm", "kernel": top_name, "achieved": hbm_achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": hbm_achieved / hbm_peak, "traffic": traffic,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel, recorded in "
                                   f"profiles/{kind}_{a.precision}_ncu.md at the current kernel sources"
                                   if traffic is not None else "no ncu capture at the current kernel sources"),
                "peak_source": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes": bytes_alg, "launch_ms": top_ms}
    # issue view: the kernel's executed warp instructions (ncu, recorded) per launch time
    # against the measured issue rate (one FP32 FMA warp instruction per scheduler and
    # clock: FP32 flops / 2 / 32)
    winst = recorded_field(kind, a.precision, "warp_inst_per_full_launch")
    issue_peak = alu["fp32_flops"] / 2.0 / 32.0 / 1e12
    if winst is not None:
        hbm_view["issue_view"] = {"achieved": winst / (top_ms * 1e-3) / 1e12, "peak": issue_peak,
                                  "unit": "T warp instructions/s", "frac": winst / (top_ms * 1e-3) / 1e12 / issue_peak,
                                  "warp_inst_per_launch": winst,
                                  "peak_source": "measured FP32 FMA rate / 64 (srfmg_alu_peaks)"}
    fp64_view = {"bound": "alu", "kernel": top_name, "achieved": achieved_tf, "peak": fp64_peak,
                 "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak, "traffic": traffic,
                 "peak_source": fp64_src,
                 "algorithmic_flops": flops, "launch_ms": top_ms}
    if prec == srfmg.FP64:
        # FP64 arithmetic: the FP64 pipe binds (about 79% busy in the segment kernels)
        roofline = dict(fp64_view, hbm_view={k: hbm_view[k] for k in ("achieved", "peak", "unit", "frac")})
    else:
        # 64-bit integer arithmetic: no FP64 work; the data movement is the path's bound
        roofline = hbm_view
    by_kind = {}
    for name, t in prof:
        k = name.split(" L")[0].replace("fx.", "")
        by_kind[k] = by_kind.get(k, 0.0) + t
    tot = sum(by_kind.values())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64" if prec != srfmg.FP64 else "f64", "data": "synthetic",
        "config": dict(workload_config(a), cta_shape=shape),
        "e2e": e2e,
        "gpu_launches": info.kernels_per_solve * a.steps,
        "plain_fp64": {"value": dist.world * N / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                       "kernels_per_solve": plain_info.kernels_per_solve,
                       "speedup_over_plain": ms_plain / ms},
        "plain_fixed": plain_fixed,
        "sr_fp64": sr64,
        "sr_levels_2": sr2,
        "adjoint": adjoint,
        "functionals_only": functionals,
        "autotune": autotune,
        "roofline": roofline,
        "kernel_share": {k: round(v / tot, 4) for k, v in sorted(by_kind.items(), key=lambda x: -x[1])},
        "clocks": clocks,
        "alu_peak": {"i64_add_per_s": alu["i64_add_per_s"], "i64_avg_ops_per_s": alu["i64_avg_ops_per_s"],
                     "fp64_tflops": alu["fp64_flops"] / 1e12, "fp32_tflops": alu["fp32_flops"] / 1e12,
                     "how": "srfmg_alu_peaks: 8 blocks x 256 threads per SM, 8 interleaved dependent chains per "
                            "thread, CUDA events, best of 5"},
    }
    err_gpu = float(np.max(np.abs(u - u_exact)))
    acc = {"err_max_vs_exact": err_gpu,
           "rel_err_max_vs_exact": err_gpu / float(np.max(np.abs(u_exact))),
           "plain_fp64_err_max_vs_exact": float(np.max(np.abs(u_plain - u_exact)))}
    if dist.rank == 0 and dist.world == 1 and not a.no_cpu_baseline:
        ref, cpu = cpu_baseline(f, M, W, b, u_exact)
        err_ref = float(np.max(np.abs(ref - u_exact)))
        acc.update({"oracle_err_max_vs_exact": err_ref,
                    "rel_maxnorm_vs_oracle": float(np.max(np.abs(u - ref)) / np.max(np.abs(ref))),
                    "at_discretization_accuracy": bool(err_gpu <= 1.5 * err_ref)})
        line["cpu_baseline"] = cpu
    line["accuracy"] = acc
    solver.close()
    del fd, ud
    torch.cuda.empty_cache()
    if not a.quick:
        # the other workloads, each with its plain FP64 baseline and accuracy flags
        a_b = argparse.Namespace(**vars(a))
        a_b.workload, a_b.batch_op = "batch", "varcoef"
        r = measure_batch(a_b, dev, dist, stream, max(3, a.steps // 4), min(a.warmup, 2), op="varcoef")
        r["config"] = dict(workload_config(a_b), segment_layout=r.pop("segment_layout"), layouts=r.pop("layouts"))
        r["metric"] = METRIC_BATCH
        line["batch"] = r
        # the Bratu workload's batch: 1024 problems of 2^12 .. 2^18 cells
        a_nb = argparse.Namespace(**vars(a))
        a_nb.workload, a_nb.batch_op, a_nb.nprob = "batch", "bratu", 1024
        r = measure_batch(a_nb, dev, dist, stream, max(5, a.steps // 4), min(a.warmup, 2), op="bratu")
        r["config"] = dict(workload_config(a_nb), segment_layout=r.pop("segment_layout"), layouts=r.pop("layouts"))
        r["metric"] = METRIC_BATCH
        line["bratu_batch"] = r
        a_r = argparse.Namespace(**vars(a))
        a_r.workload, a_r.log2n, a_r.precision = "bratu", 26, "mixed"
        r = measure_single(a_r, dev, dist, stream, "bratu", "mixed", max(5, a.steps // 2), min(a.warmup, 3))
        r["config"] = dict(workload_config(a_r), cta_shape=r.pop("cta_shape"))
        r["metric"] = METRIC_BRATU
        line["bratu"] = r
        if dist.rank == 0 and dist.world == 1 and not a.no_cpu_baseline:
            line["cpu_baseline_allcores"] = cpu_baseline_allcores(M, W, b)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()


def measure_single(a, dev, dist, stream, kind, precision, steps, warmup, full=True, oracle_check=True):
    """One problem of the variable-coefficient ("varcoef") or Bratu ("bratu")
    workload at N = 2^a.log2n: the SR solve in `precision` ("mixed" or
    "fp64"); with `full`, the plain FP64 stored-grid solve of the same problem,
    the solve from host memory, the longest launch's FP64 roofline and, with
    `oracle_check`, the oracle's solve for the accuracy flags.  Returns a dict."""
    import torch
    from paper_1207_6720_gb300 import srfmg, workloads

    M, W, b = a.log2n, a.segment_width, a.buffer_width
    N = 1 << M
    vcoef = kind == "varcoef"
    mixed = precision == "mixed"
    prec = srfmg.MIXED if mixed else srfmg.FP64
    if vcoef:
        f, u_exact, log_a = workloads.varcoef_series(M, 16, seed=1)
        kw = dict(op=srfmg.VARCOEF, nu1=1, nu2=1)
        flops_table = FLOPS_PER_CELL_VARCOEF
    else:
        f, u_exact, _ = workloads.bratu_series(M, 16, seed=1, lam=a.lam)
        kw = dict(op=srfmg.BRATU, lambda_=a.lam, nu1=2, nu2=1)
        flops_table = FLOPS_PER_CELL_BRATU_MX if mixed else FLOPS_PER_CELL_BRATU
    fd = torch.from_numpy(f).to(dev)
    ud = torch.empty_like(fd)
    log_a_d = torch.from_numpy(log_a).to(dev) if vcoef else None
    solver, shape = tuned_solver(srfmg, M, dev, reps=2, coef=log_a_d, segment_width=W, buffer_width=b,
                                 precision=prec, **kw)
    info = solver.info()
    sampler = ClockSampler(dev)
    sampler.start()
    ms = dist.max(time_solves(solver, fd, ud, steps, warmup, dist, stream))
    clocks = sampler.stop()
    u = ud.cpu().numpy()
    out = {"value": dist.world * N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "warmup": warmup, "precision": precision, "N": N, "gpu_launches": info.kernels_per_solve * steps,
           "clocks": clocks, "cta_shape": shape}
    if full:
        alu_peak(dev)
        plain, _ = tuned_solver(srfmg, M, dev, reps=2, coef=log_a_d, n_sr_levels=0, **kw)
        ms_plain = dist.max(time_solves(plain, fd, ud, max(5, steps // 4), min(warmup, 3), dist, stream))
        u_plain = ud.cpu().numpy()
        plain.close()
        fh = torch.from_numpy(f).pin_memory()
        uh = torch.empty(N, dtype=torch.float64).pin_memory()
        fh_np, uh_np = fh.numpy(), uh.numpy()
        solver.solve_host(fh_np, uh_np, stream=stream)
        dist.barrier()
        e2e_steps = max(3, steps // 10)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solver.solve_host(fh_np, uh_np, stream=stream)
        dt_e2e = dist.max((time.perf_counter() - t0) / e2e_steps)
        prof = solver.profile(fd, torch.empty_like(fd), nsolves=3, stream=stream)
        torch.cuda.synchronize()
        # the roofline kernel: the longest launch of the streaming kernels (the
        # one-block coarse tail and the right-hand-side hierarchy excluded)
        top_name, top_ms = max(((nm, t) for nm, t in prof if nm.split(" L")[0].replace("fx.", "") in STREAMING),
                               key=lambda x: x[1])
        kname, lvl = top_name.split(" L")
        kname = kname.replace("fx.", "")
        cells = 1 << int(lvl)
        flops = flops_table.get(kname, 0.0) * cells
        achieved_tf = flops / (top_ms * 1e-3) / 1e12
        peaks = measured_peaks()
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        fixed_vc = vcoef and mixed
        bytes_alg = (BYTES_PER_CELL_VC_FX if fixed_vc else BYTES_PER_CELL).get(kname, 0.0) * cells
        fp64_peak, fp64_src = fp64_peak_tflops()
        hbm_achieved = bytes_alg / (top_ms * 1e-3) / 1e9
        if fixed_vc:       # 64-bit fixed point: no FP64 work; the data movement is the path's bound
            roof = {"bound": "hbm", "kernel": top_name, "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak, "traffic": None,
                    "peak_source": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback",
                    "algorithmic_bytes": bytes_alg, "launch_ms": top_ms}
        else:
            roof = {"bound": "alu", "kernel": top_name, "achieved": achieved_tf,
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak, "traffic": None,
                    "peak_source": fp64_src + " (FP64 operations of the method per cell; exponential and "
                                              "reciprocal counted as one operation)",
                    "algorithmic_flops": flops, "launch_ms": top_ms,
                    "hbm_view": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": hbm_achieved / hbm_peak}}
        out.update({
            "e2e": {"value": dist.world * N / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": int(f.nbytes),
                    "d2h_bytes_per_step": int(uh_np.nbytes)},
            "plain_fp64": {"value": dist.world * N / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                           "speedup_over_plain": ms_plain / ms,
                           "err_max_vs_exact": float(np.max(np.abs(u_plain - u_exact)))},
            "roofline": roof,
        })
    err = float(np.max(np.abs(u - u_exact)))
    acc = {"err_max_vs_exact": err, "rel_err_max_vs_exact": err / float(np.max(np.abs(u_exact)))}
    if dist.rank == 0 and dist.world == 1 and not a.no_cpu_baseline and full and oracle_check:
        import oracle
        if vcoef:
            p = oracle.sr_params(M, W, b, nRS=1, op="varcoef", coef=np.exp(log_a))
        else:
            p = oracle.sr_params(M, W, b, nRS=1, nu1=2, nu2=1, op="bratu", lam=a.lam)
        t0 = time.perf_counter()
        ref = oracle.fmg_v(p, f)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": N / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"one serial solve of the full N=2^{M} workload (C oracle, "
                                         f"serial SR with the finest level never stored)"}
        err_ref = float(np.max(np.abs(ref - u_exact)))
        rel_or = float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))
        acc.update({"oracle_err_max_vs_exact": err_ref, "rel_maxnorm_vs_oracle": rel_or,
                    "at_discretization_accuracy": bool(err <= 1.5 * err_ref),
                    "parity_vs_oracle_1e-10": bool(rel_or <= 1e-10)})
        if err_ref < 1e-11 * float(np.max(np.abs(u_exact))) * 100:
            acc["note"] = ("rounding-limited size: the O(h^2) truncation error is below the FP64 rounding of "
                           "either solve, so the error against the exact solution compares roundings; the "
                           "parity flag is the accuracy criterion here")
    out["accuracy"] = acc
    solver.close()
    del fd, ud
    torch.cuda.empty_cache()
    return out


def run_gpu_bratu(a):
    """The Bratu or variable-coefficient workload as its own JSON line."""
    import torch
    dist = Dist(a.gpus, use_cuda=True)
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    r = measure_single(a, dev, dist, stream, a.workload, a.precision, a.steps, a.warmup, full=not a.only_solve)
    metric = METRIC_VARCOEF if a.workload == "varcoef" else METRIC_BRATU
    line = {"metric": metric, "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": dist.world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": r.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("int64" if a.workload == "varcoef" else "f64+f32") if a.precision == "mixed" else "f64",
            "data": "synthetic", "config": dict(workload_config(a), cta_shape=r.pop("cta_shape"))}
    for k in ("steps", "warmup", "precision", "N"):
        r.pop(k)
    line.update(r)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()


def measure_batch(a, dev, dist, master, steps, warmup, op="varcoef", tune=True, full=True):
    """Many independent problems of uneven sizes (8192 by default, N = 2^m with
    m ~ U{10..20}): one srfmg group (a batched plan per size, all replayed as
    one CUDA graph), one group solve per step, in the mixed precision; with
    `full`, also the group of plain FP64 stored-grid plans on the same problems,
    the group solve from host memory, the longest launch's roofline and the
    accuracy of a sample against the exact solution and the oracle.  Returns
    the measurement as a dict (the workload's JSON line without its header)."""
    import torch
    from paper_1207_6720_gb300 import srfmg, workloads

    nl = op == "bratu"
    sizes = workloads.batch_sizes(a.nprob, 12, 18, seed=11) if nl else workloads.batch_sizes(a.nprob, 10, 20, seed=11)
    classes = {}
    for k, m in enumerate(sizes):
        classes.setdefault(int(m), []).append(k + 1000)       # problem k's series seed
    total = int(sum(len(v) << m for m, v in classes.items()))
    vc = op == "varcoef"
    # the packed layout: by size, then by index (srfmg_group_offsets); log a per plan
    fparts, laparts = [], []
    for m in sorted(classes):
        if vc:
            fm, lam = workloads.varcoef_series_batch(m, classes[m], 32, dev)
            fparts.append(fm)
            laparts.append(lam)
        elif nl:
            fparts.append(workloads.bratu_series_batch(m, classes[m], 16, a.lam, dev))
        else:
            fparts.append(workloads.sine_series_batch(m, classes[m], 32, dev)[0])
    fd = torch.cat(fparts)
    del fparts
    la_d = torch.cat(laparts) if vc else None
    del laparts
    ud = torch.empty_like(fd)
    assert fd.numel() == total == int(srfmg.group_offsets(sizes)[-1])
    torch.cuda.synchronize()
    kw_op = (dict(op=srfmg.VARCOEF) if vc else
             dict(op=srfmg.BRATU, lambda_=a.lam, nu1=2, nu2=1) if nl else {})

    def make(prec, nRS, tune_reps):
        kw = dict(precision=prec, n_sr_levels=nRS, **kw_op)
        if nRS:
            kw.update(segment_width=4096, buffer_width=8)
        g = srfmg.Group(sizes, device=dev, tune=tune_reps, **kw)
        if vc:       # every plan's coefficient from its part of the packed log a
            o = 0
            for mb in g.members():
                cnt = mb.batch * (mb.n + 1)
                mb.set_coefficient(la_d[o:o + cnt], stream=master)
                o += cnt
            assert o == la_d.numel()
        return g

    def timed(group, nsteps, nwarm):
        for _ in range(nwarm):
            group.solve(fd, ud, stream=master)
        torch.cuda.synchronize()
        dist.barrier()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(master)
        for _ in range(nsteps):
            group.solve(fd, ud, stream=master)
        t1.record(master)
        t1.synchronize()
        torch.cuda.synchronize()
        dist.barrier()
        return t0.elapsed_time(t1) / nsteps

    tune_reps = 3 if tune else 0
    t_create = time.perf_counter()
    group = make(srfmg.MIXED, 1, tune_reps)
    t_create = time.perf_counter() - t_create
    members = group.members()
    launches = sum(mb.info().kernels_per_solve for mb in members)
    layouts = {str(mb.n.bit_length() - 1): [mb.params.segment_width, mb.params.buffer_width,
                                            mb.info().coarse_tail_level] for mb in members}
    sampler = ClockSampler(dev)
    sampler.start()
    ms = dist.max(timed(group, steps, warmup))
    clocks = sampler.stop()
    value = dist.world * total / (ms * 1e-3)
    out = {"value": value, "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "unknowns_per_step": total, "group_create_s": t_create, "gpu_launches": launches * steps,
           "clocks": clocks,
           "segment_layout": ("autotuned per size: (W, b) by srfmg_autotune, then the CTA shape by "
                              "srfmg_autotune_shape, 3 timed solves per candidate; layouts: [W, b, coarse tail level]"
                              if tune else "min(4096, N/4) cells, buffer 8"),
           "layouts": layouts}
    # accuracy sample: the first problem of every size against its exact solution
    samples = {}
    worst = 0.0
    for mb in members:
        m = mb.n.bit_length() - 1
        if m in samples:
            continue
        o = int(mb.offset)
        u0 = ud[o:o + mb.n].cpu().numpy()
        if vc:
            f0, ue, la0 = workloads.varcoef_series(m, 32, classes[m][0])
        elif nl:
            f0, ue, _ = workloads.bratu_series(m, 16, classes[m][0], a.lam)
            la0 = None
        else:
            f0, ue, _ = workloads.sine_series(m, 32, classes[m][0])
            la0 = None
        samples[m] = (f0, ue, la0, u0, mb.params.segment_width, mb.params.buffer_width)
        worst = max(worst, float(np.max(np.abs(u0 - ue))))
    if full:
        # end to end: the whole group through srfmg_group_solve_host from pinned host buffers
        fh = fd.cpu().pin_memory()
        uh = torch.empty(total, dtype=torch.float64).pin_memory()
        group.solve_host(fh.numpy(), uh.numpy(), stream=master)
        t0 = time.perf_counter()
        group.solve_host(fh.numpy(), uh.numpy(), stream=master)
        dt_e2e = dist.max(time.perf_counter() - t0)
        out["e2e"] = {"value": dist.world * total / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": total * 8,
                      "d2h_bytes_per_step": total * 8}
        del fh, uh
        # roofline view: the longest launch of the largest size's plan
        big = max(members, key=lambda mb: mb.n * mb.batch)
        o = int(big.offset)
        prof = big.profile(fd[o:o + big.n * big.batch], torch.empty(big.n * big.batch, dtype=torch.float64,
                                                                    device=fd.device), nsolves=2, stream=master)
        torch.cuda.synchronize()
        top_name, top_ms = max(((nm, t) for nm, t in prof if nm.split(" L")[0].replace("fx.", "") in STREAMING),
                               key=lambda x: x[1])
        kind, lvl = top_name.split(" L")
        kind = kind.replace("fx.", "")
        # (the Bratu problem's kernels are the FP64 ones: 8-byte u; their bound is the FP64 pipe,
        # reported for the single problem; here the data-movement view)
        bytes_alg = (BYTES_PER_CELL_VC_FX if vc else BYTES_PER_CELL).get(kind, 0.0) * big.batch * (1 << int(lvl))
        peaks = measured_peaks()
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        out["roofline"] = {"bound": "hbm", "kernel": f"{top_name} (batch of {big.batch})",
                           "achieved": bytes_alg / (top_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                           "frac": bytes_alg / (top_ms * 1e-3) / 1e9 / hbm_peak, "traffic": None,
                           "peak_source": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback",
                           "launch_ms": top_ms}
    group.close()
    if full:
        plain = make(srfmg.FP64, 0, 0)
        ms_plain = dist.max(timed(plain, max(2, steps // 2), 1))
        plain.close()
        first = {}
        for mb in members:
            first.setdefault(mb.n.bit_length() - 1, int(mb.offset))
        err_plain = max(float(np.max(np.abs(ud[o:o + (1 << m)].cpu().numpy() - samples[m][1])))
                        for m, o in first.items())
        out["plain_fp64"] = {"value": dist.world * total / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                             "speedup_over_plain": ms_plain / ms, "err_max_vs_exact_sample": err_plain}
    acc = {"err_max_vs_exact_sample": worst, "sample": "first problem of each size"}
    if dist.rank == 0 and dist.world == 1 and not a.no_cpu_baseline and full:
        import oracle
        refs = {}
        t0 = time.perf_counter()
        reps = 0
        while True:
            for m, (f0, ue, la0, u0, W, b) in samples.items():
                okw = (dict(op="varcoef", coef=np.exp(la0)) if vc else
                       dict(op="bratu", lam=a.lam, nu1=2, nu2=1) if nl else {})
                refs[m] = oracle.fmg_v(oracle.sr_params(m, W, b, **okw), f0)
            reps += 1
            if time.perf_counter() - t0 > 5.0 or reps >= 10:
                break
        dt = time.perf_counter() - t0
        n_sample = sum(1 << m for m in samples)
        out["cpu_baseline"] = {"value": reps * n_sample / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{reps} x one problem of each size ({n_sample} unknowns) "
                                         f"with the serial C oracle"}
        ok = all(np.max(np.abs(u0 - ue)) <= 1.5 * np.max(np.abs(refs[m] - ue))
                 for m, (f0, ue, la0, u0, W, b) in samples.items())
        acc.update({"rel_maxnorm_vs_oracle_sample": max(
            float(np.max(np.abs(u0 - refs[m])) / np.max(np.abs(refs[m])))
            for m, (f0, ue, la0, u0, W, b) in samples.items()),
            "at_discretization_accuracy_sample": bool(ok)})
    out["accuracy"] = acc
    del fd, ud, la_d
    torch.cuda.empty_cache()
    return out


def run_gpu_batch(a):
    """The batch workload as its own JSON line."""
    import torch
    dist = Dist(a.gpus, use_cuda=True)
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    master = torch.cuda.current_stream()
    r = measure_batch(a, dev, dist, master, a.steps, a.warmup, op=a.batch_op, tune=not a.no_tune,
                      full=not a.only_solve)
    cfg = workload_config(a)
    cfg["segment_layout"] = r.pop("segment_layout")
    cfg["layouts"] = r.pop("layouts")
    line = {"metric": METRIC_BATCH, "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": dist.world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": r.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": cfg}
    r.pop("steps")
    r.pop("warmup")
    line.update(r)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()


def main():
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_gpu_batch(a)
    elif a.workload in ("bratu", "varcoef"):
        run_gpu_bratu(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
