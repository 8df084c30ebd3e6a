#!/usr/bin/env python
"""Benchmark: synchronous Parareal on the 3D heat workload, one JSON line.

Workload (default "heat3d_mixed"): u_t = Laplace(u) on the unit cube, 256^3
interior grid, zero Dirichlet boundary, N = 128 slices, F = 64 explicit-Euler
7-point steps per slice at dt = 0.15 h^2 in FP32 (FP64 input and output), G =
one implicit Euler step per slice solved by CG in FP64 (rtol 1e-7), the
correction and the stopping test in FP64, u0 = N(0,1) noise smoothed by three
damped-Jacobi sweeps (seeded), stop when max_i ||lam_i^k - lam_i^{k-1}||_inf
< 1e-5.  One "step" = one complete Parareal solve (predictor, batched fine
sweeps, coarse sweeps with the fused correction and test) to the tolerance.
Beside it the line carries the same solve with FP64 fine steps (time to 1e-5
of both, and both errors against the FP64 serial fine solution) and the GPU
serial fine solve.  --workload selects the other workloads (2D FP64, async,
adjoint, trapezoidal F).

metric: fine GLUP/s = fine cell updates executed / wall time of the solves.

Multi-GPU (torchrun): replicas only -- every rank solves its own copy of the
workload; value = units of all ranks / max-over-ranks time (weak scaling).
--impl reference times the FP64 CPU oracle on a bounded sample instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "heat2d_cn": "2D heat 512x512, N=32 slices, F=100 trapezoidal-rule (Crank-Nicolson) steps "
                 "(dt=4h^2, each solved by CG to rtol 1e-12 from the current state), G=1 implicit "
                 "Euler step by CG (rtol 1e-10), FP64, sync Parareal, tol 1e-6",
    "heat2d_inverse_async": "2D inverse heat 512x512, variable kappa, N=32, F=128: loss + gradient "
                            "wrt u0 and kappa through the logged asynchronous run (tol 1e-8) by "
                            "device replay and reverse pass over the event graph, FP64",
    "heat2d_cn_async": "the 2D heat 512x512 N=32 trapezoidal-F problem (Table 1's F and G) solved "
                       "by the asynchronous persistent kernel (no injected delays) next to the "
                       "synchronous solve, tol 1e-6",
    "heat2d_explicit": "2D heat 1024x1024, N=64 slices, F=256 explicit 5-pt steps (dt=0.2h^2), "
                       "G=1 implicit Euler step by FP64 CG (rtol 1e-10) preconditioned by 16 FP32 "
                       "Chebyshev steps, FP64, sync Parareal, tol 1e-10",
    "heat3d_mixed": "3D heat 256^3, N=128 slices, F=64 explicit 7-pt steps (dt=0.15h^2), "
                    "G=implicit Euler by FP64 CG (rtol 1e-7) preconditioned by 12 FP32 Chebyshev "
                    "steps, FP32 fine / FP64 coarse vs plain FP64, sync, time to 1e-5",
    "heat1d_thomas": "1D heat 1023 pts, N=16 slices, F=100 implicit Euler steps, G=1 step, both "
                     "by the batched partition Thomas/PCR solver, FP64, sync, tol 1e-10",
    "heat2d_async": "the 2D heat 1024x1024 N=64 FP64 problem solved by the asynchronous persistent "
                    "kernel (no injected delays) next to the synchronous solve, tol 1e-10",
    "heat3d_varkappa_async": "3D variable-kappa heat 192^3, N=256, F=32 explicit 7-pt steps, FP32 "
                             "fine / FP64 coarse, async with seeded publish delays 0-4 fine-step "
                             "units vs sync, tol 1e-5",
    "heat2d_inverse": "2D inverse heat 512x512, variable kappa, N=32, F=128, K=6 Parareal "
                      "iterations: loss + discrete-adjoint gradient wrt u0 and kappa, FP64",
}
# FP64-pipe operations per fine cell update (DADD/DMUL/DFMA each one issue slot).
# Constant kappa, explicit: the library runs the scaled form (states carried as
# u / rx^j, which removes the x multiplier): 1D 1 DADD + 1 DFMA, 2D 2 DADD + 2 DFMA,
# 3D 3 DADD + 3 DFMA, plus one DMUL on the steps that return to u (every R steps and
# the last one, R = floor(100 / log10(1/rx))), in the batched and the asynchronous
# kernels alike.  Plain form (scaled=False): 1 DMUL + d DADD + d DFMA.  Variable kappa:
# 1 DMUL + 2d DFMA.  1D implicit step by the partition solver: 2 (forward) + 1 (back)
# + 2 (rebuild).
def fp64_ops_per_lup(p, scaled=True):
    dim = p["dim"]
    if p.get("f_scheme") == "implicit":
        return 5.0
    if p.get("kappa") is not None or not scaled:
        return 1.0 + 2 * dim
    rx = p["dt"] / (1.0 / (p["n"][0] + 1)) ** 2
    R = max(1, int(math.floor(100.0 / math.log10(1.0 / rx))))
    return 2.0 * dim + math.ceil(p["f_steps"] / R) / p["f_steps"]


# Trapezoidal F in 2D/3D: per CG iteration and point, the operator scaled by 1/R_x
# (d DADD + d DFMA) plus 5 DFMA (p.q, x, r, r.r, p); per fine step and point, the
# right-hand side (explicit form: 1 DMUL + d DADD + d DFMA), the start residual
# (the unscaled operator and b - Ax) and its two norms.
CN_OPS_PER_CG_POINT = {2: 9, 3: 11}
CN_OPS_PER_LUP = {2: 13, 3: 17}
NOMINAL_FP64_OPS = 625.0  # G FP64-pipe ops/s: 1.25 TFLOP/s nominal / 2 flops per DFMA
# DRAM bytes (read + write) per cell update of the dominant kernel, from one ncu capture
# of the current kernel; None where no capture of the current kernel exists.
# (profiles/step2d_fp64_heat2d_1024x1024.md: 1016.3 MB for 63 x 1048576 updates.)
NCU_TRAFFIC_PER_LUP = {"heat2d_explicit": 1016.3e6 / (63 * 1048576),
                       # profiles/step3d_tma2_fp32_heat3d_256cubed_N4.md: 520.4 MB for one
                       # two-step pass over 4 x 256^3 points (2 updates each)
                       "heat3d_mixed": 520.4e6 / (2 * 4 * 256 ** 3)}
# The coarse CG kernel's DRAM bytes over its algorithmic bytes (pcg_pass_costs), from
# one ncu capture of every cg_kernel launch of a small run of the same workload
# (profiles/pcg_cg_kernel_heat3d_256cubed_N4.md: 353.37 GB for 350.31 GB algorithmic,
# 10 solves and 78 iterations at 256^3, the solve kernels with their correction
# kernels); traffic per launch = ratio x the bench's algorithmic bytes per launch.
NCU_COARSE_TRAFFIC_RATIO = {"heat3d_mixed": 353.37 / 350.31}


def cost_model_sync(p, st, ms_per_solve):
    """The cost model of §4.1 evaluated on one measured synchronous solve.

    C_F: one iteration's fine phase (every active slice's F runs at once on the
    device, the analogue of one processor per slice applying F); C_G: one
    coarse solve.  Aubanel's pipelined cost p C_G + k (C_F + C_G) assumes the
    coarse chain of an iteration overlaps the next fine phase; Proposition 2
    adds an average non-overlapped overhead C_bar per processor and iteration:
        C^(k) = p C_G + k (C_F + C_G + (p - 1 - (k + 1) / 2) C_bar),
    solved here for C_bar from the measured time.  On one device the coarse
    sweep does not overlap the fine phase, so C_bar comes out close to C_G.
    """
    k, N = int(st["iterations"]), int(p["N"])
    solves = max(int(st["coarse_solves"]), 1)
    C_F = st["t_fine_ms"] / max(k, 1)
    C_G = st["t_coarse_ms"] / solves
    ideal = N * C_G + k * (C_F + C_G)
    denom = k * (N - 1) - k * (k + 1) / 2
    return {"p": N, "k": k, "C_F_ms": C_F, "C_G_ms": C_G, "coarse_solves": solves,
            "aubanel_ms": ideal, "measured_ms": ms_per_solve,
            "C_bar_ms": (ms_per_solve - ideal) / denom if denom > 0 else None,
            "serial_fine_model_ms": N * C_F}


def sync_delay_ms(table, unit_ns, k, N):
    """Time the injected publication delays add to a synchronous run of k
    iterations: version j+1 of slice i is published with delay
    table[i-1, j % cols] units, and in the synchronous sweep every published
    correction sits on the critical path (the next slice's coarse solve
    waits for it), so the delays of the updated slices add up."""
    cols = table.shape[1]
    units = sum(float(table[i - 1, j % cols]) for j in range(k) for i in range(j + 1, N + 1))
    return units * unit_ns / 1e6


def apr_cost(p, kappa, C_F, C_G):
    """Proposition 3 (§4.1): cost of kappa(k~) asynchronous iterations with one
    processor per slice and communication fully overlapped,
        C~ = p C_G + kappa (C_F + C_G)."""
    return p * C_G + kappa * (C_F + C_G)


def cost_model_async(log, N, t_ms):
    """Per-update costs of an asynchronous run read from its event log (§4.1,
    Proposition 3 charges kappa (C_F + C_G) per processor): the mean duration
    of the updates without a coarse solve (F only) and with one (F + G), and
    kappa(k~) = max_i k_i.  Durations run from the update's start to the
    version's visibility, so injected delays are included."""
    f_only = [(e.t_end - e.t_start) / 1e6 for e in log if e.vG == e.vF]
    f_g = [(e.t_end - e.t_start) / 1e6 for e in log if e.vG != e.vF]
    k_i = {}
    for e in log:
        k_i[e.slice] = max(k_i.get(e.slice, 0), e.version)
    mean = lambda v: sum(v) / len(v) if v else None
    return {"p": N, "kappa": max(k_i.values()) if k_i else 0, "updates": len(log),
            "update_F_ms": mean(f_only), "update_FG_ms": mean(f_g),
            "n_F_only": len(f_only), "n_FG": len(f_g), "measured_ms": t_ms}


def cost_models(log, N, t_async, p, sync_stats, t_sync):
    """Both cost models on one problem, plus Proposition 3's estimate of the
    asynchronous time from the synchronous run's C_F and C_G (the model's one
    processor per slice, each F as fast as one batched fine phase)."""
    a = cost_model_async(log, N, t_async)
    sm = cost_model_sync(p, sync_stats, t_sync)
    a["prop3_ms"] = apr_cost(N, a["kappa"], sm["C_F_ms"], sm["C_G_ms"])
    return {"async": a, "sync": sm}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heat3d_mixed", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-fp64", action="store_true",
                    help="mixed workloads: skip the FP64 comparison solve (tuning sweeps)")
    ap.add_argument("--profile", action="store_true",
                    help="run exactly one solve and nothing else (for ncu launch lists)")
    ap.add_argument("--g-rtol", type=float, default=None,
                    help="override the coarse CG tolerance of the workload")
    ap.add_argument("--grid", default=None,
                    help="override the grid, e.g. 160,160,160 (small cases for ncu captures)")
    ap.add_argument("--slices", type=int, default=None, help="override N (small cases)")
    ap.add_argument("--pipeline", action="store_true",
                    help="overlap F of iteration k+1 with the coarse sweep of iteration k")
    ap.add_argument("--chunks", type=int, default=8, help="slice chunks per pipelined F batch")
    ap.add_argument("--g-cheb", type=int, default=None,
                    help="coarse CG preconditioned by this many FP32 Chebyshev steps (0 = plain "
                         "CG; default: the workload's setting)")
    ap.add_argument("--f-per-pass", type=int, default=2, choices=[1, 2],
                    help="TMA-fed FP32 fine steps per pass over the state (temporal blocking)")
    ap.add_argument("--g-cg", type=int, default=0, choices=[0, 1, 2],
                    help="unpreconditioned coarse CG recurrence: 0 automatic, 1 textbook, "
                         "2 single-reduction")
    ap.add_argument("--ctas-per-slice", type=int, default=0,
                    help="async workloads: CTAs per slice team (0 = automatic)")
    ap.add_argument("--lazy", action="store_true",
                    help="async workloads: skip re-updates that a newer input will supersede")
    ap.add_argument("--verify", action="store_true",
                    help="async workloads: confirm the stop by the fixed-point residual")
    ap.add_argument("--cg-bps", type=int, default=0,
                    help="CG blocks per SM under the pipeline (0 = automatic)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_aggregate(units, seconds, world, device="cpu"):
    """Whole-job throughput of independent replicas: (sum of units over ranks) /
    (max time over ranks).  Returns (units per second, max seconds)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        u = torch.tensor([float(units)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        seconds, units = float(t.item()), float(u.item())
    return units / seconds, seconds


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


G_RTOL_OVERRIDE = None
SIZE_OVERRIDE = {}


def preset_args(name):
    """(preset name, overrides) of a workload: the synthetic recipe and the
    size/tolerance overrides given on the command line."""
    base = {"heat2d_async": "heat2d_explicit", "heat2d_cn_async": "heat2d_cn",
            "heat2d_inverse_async": "heat2d_inverse"}.get(name, name)
    over = dict(SIZE_OVERRIDE)
    if G_RTOL_OVERRIDE is not None:
        over["g_rtol"] = G_RTOL_OVERRIDE
    return base, over


def problem_of(name):
    from synthetic import preset
    base, over = preset_args(name)
    return preset(base, "full", **over)


def bench_config(args, p, world=1):
    """`config` of the bench line; the reference arm prints the same keys."""
    cfg = {"workload": WORKLOADS[args.workload], "grid": list(p["n"]), "N": p["N"],
           "f_steps": p["f_steps"], "tol": p.get("tol"), "g_rtol": p.get("g_rtol"),
           "f_prec": p.get("f_prec", 64),
           "parallelism": "replicas" if world > 1 else "1 GPU",
           "schedule": ("pipelined (F of k+1 overlaps the sweep of k)"
                        if getattr(args, "pipeline", False) else "plain"),
           "coarse_solver": ("Thomas (partition tridiagonal solver)"
                             if p.get("g_solver") == "thomas" else
                             "CG preconditioned by %d FP32 Chebyshev steps" % args.g_cheb
                             if args.g_cheb else "CG"),
           "l2": "inputs larger than L2 (trajectory %.2f GB + workspaces)" % (
               (p["N"] + 1) * math.prod(p["n"]) * 8 / 1e9)}
    return cfg


def problem_struct(pr, p, u0, kappa=None, **over):
    """pr_problem for a preset dict (T0 = 0, T = N * f_steps * dt)."""
    kw = dict(dim=p["dim"], n=p["n"], T0=0.0, T=p["N"] * p["f_steps"] * p["dt"], N=p["N"],
              u0=u0, kappa=kappa,
              f_scheme={"implicit": pr.PR_IMPLICIT_EULER, "cn": pr.PR_CRANK_NICOLSON}.get(
                  p.get("f_scheme"), pr.PR_EXPLICIT_EULER),
              f_steps=p["f_steps"], f_prec=p.get("f_prec", 64),
              g_solver=pr.PR_SOLVER_THOMAS if p.get("g_solver") == "thomas" else pr.PR_SOLVER_CG,
              g_rtol=p.get("g_rtol", 1e-10), tol=p.get("tol", 0.0),
              f_rtol=p.get("f_rtol") or 0.0)
    kw.update(over)
    return pr.make_problem(**kw)


# ---------------------------------------------------------------- CPU baseline
# The FP64 oracle (numpy, as it stands) timed on all host cores: a pool of
# spawned processes, one slice per process (the slices' fine propagations are
# independent, Algorithm 1), each single-threaded.  Spawned, not forked: a
# child forked after the first CUDA call can hang.
_ORACLE = {}


def _oracle_init(name, over):
    from oracle import heat
    from synthetic import preset
    _ORACLE["p"] = preset(name, "full", **over)
    _ORACLE["heat"] = heat


def _oracle_fine_task(args):
    """One slice's F, `steps` fine steps of the full grid; returns (LUPs, t0, t1)."""
    import numpy as np
    seed, steps = args
    p, heat = _ORACLE["p"], _ORACLE["heat"]
    P = heat.Propagators(dict(p, f_steps=steps))
    x = p["u0"] + 0.01 * np.random.default_rng(seed).standard_normal(p["u0"].shape)
    t0 = time.time()
    P.F(x)
    t1 = time.time()
    return steps * int(np.prod(p["n"])), t0, t1


def _oracle_cg_task(iters):
    """`iters` iterations of the oracle's coarse CG on the full grid; returns seconds."""
    p, heat = _ORACLE["p"], _ORACLE["heat"]
    P = heat.Propagators(dict(p, g_rtol=0.0, g_maxit=iters))
    t0 = time.perf_counter()
    P.G(p["u0"])
    return time.perf_counter() - t0


class OraclePool:
    """All host cores running the oracle, one slice per spawned process."""

    def __init__(self, name, over, cores=None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                 initargs=(name, dict(over)))

    def fine(self, steps):
        """Every core propagates one slice by `steps` fine steps at once; returns
        (GLUP/s over the wall time of the parallel region, seconds, LUPs)."""
        res = self.pool.map(_oracle_fine_task, [(s, steps) for s in range(self.cores)],
                            chunksize=1)
        lups = sum(r[0] for r in res)
        wall = max(r[2] for r in res) - min(r[1] for r in res)
        return lups / wall / 1e9, wall, lups

    def cg_iteration_s(self, iters=2):
        """Seconds per oracle coarse-CG iteration (one core)."""
        return self.pool.apply(_oracle_cg_task, (iters,)) / iters

    def close(self):
        self.pool.terminate()
        self.pool.join()


def host_cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def oracle_sample_steps(p):
    """Fine steps per slice of one bounded oracle sample (about a second or two of
    numpy per core at the workload's full grid)."""
    M = 1
    for v in p["n"]:
        M *= v
    if p.get("f_scheme") == "cn":
        return 2
    return max(1, min(p["f_steps"], int(2.5e7 // M)))


def oracle_time_to_tol_s(p, fine_s_per_step_slice, cg_it_s, cores, k, cg_iterations):
    """Time of the oracle's synchronous Parareal solve on `cores` host cores,
    extrapolated (labelled as such): the fine phase of iteration j runs the
    N - j active slices' F spread over the cores, the coarse sweep and the
    predictor are sequential CG solves.  Work counts (k, CG iterations) are the
    GPU run's; per-unit costs are the oracle's, measured on this host."""
    N, nf = p["N"], p["f_steps"]
    fine = sum(math.ceil((N - j) / cores) for j in range(k)) * nf * fine_s_per_step_slice
    return fine + cg_iterations * cg_it_s


def cpu_baseline_leg(name, p, over, gpu_stats=None):
    """cpu_baseline object of the bench line: the oracle's fine GLUP/s on all
    host cores (bounded sample), plus the extrapolated oracle time-to-tolerance
    when the GPU run's work counts are given."""
    t_start = time.perf_counter()
    steps = oracle_sample_steps(p)
    pool = OraclePool(name, over)
    try:
        pool.fine(1)                              # warm-up: spawn, imports, inputs
        v, wall, lups = pool.fine(steps)
        out = {"value": v, "unit": "GLUP/s", "cores": pool.cores, "kind": "oracle",
               "cpu": host_cpu_model(),
               "sample": "oracle F (numpy FP64, one single-threaded process per core) on %d "
                         "slices x %d fine steps of the full %s grid at once, %.1f s" % (
                             pool.cores, steps, "x".join(map(str, p["n"])), wall)}
        if gpu_stats is not None and p.get("g_solver") != "thomas":
            cg_it = pool.cg_iteration_s(2)
            per_step_slice = wall / steps     # every core ran one slice of `steps` steps
            k, cgi = gpu_stats["iterations"], gpu_stats["cg_iterations"]
            t = oracle_time_to_tol_s(p, per_step_slice, cg_it, pool.cores, k, cgi)
            out["time_to_tol_s_extrapolated"] = t
            out["time_to_tol_basis"] = (
                "extrapolated: %d iterations, %d coarse CG iterations (the GPU run's counts); "
                "oracle F %.3f s per fine step and slice (cores in parallel), oracle CG "
                "%.3f s per iteration (one core; the sweep is sequential)" % (
                    k, cgi, per_step_slice, cg_it))
    finally:
        pool.close()
    out["leg_s"] = time.perf_counter() - t_start
    return out


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle as it stands, on all host cores, on a
    bounded sample of the same workload per step (every core propagates one
    slice by a few fine steps of the full grid)."""
    if rank != 0:
        return 0
    p = problem_of(args.workload)
    base, over = preset_args(args.workload)
    steps = oracle_sample_steps(p)
    pool = OraclePool(base, over)
    try:
        pool.fine(1)
        for _ in range(args.warmup):
            pool.fine(steps)
        tot_t, tot_l = 0.0, 0
        for _ in range(args.steps):
            _, wall, lups = pool.fine(steps)
            tot_t += wall
            tot_l += lups
        cores = pool.cores
    finally:
        pool.close()
    v = tot_l / tot_t / 1e9
    sample = ("oracle F (numpy FP64, one single-threaded process per core) on %d slices x %d "
              "fine steps of the full %s grid at once per step" % (
                  cores, steps, "x".join(map(str, p["n"]))))
    out = {"impl": "reference", "metric": "fine GLUP/s", "value": v, "unit": "GLUP/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "config": bench_config(args, p, world),
           "cpu_baseline": {"value": v, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
                            "cpu": host_cpu_model(), "sample": sample},
           "e2e": {"value": v, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def apply_coarse_options(pr, ctx, args):
    if args.g_cheb:
        pr.parareal_set_option(ctx, pr.PR_OPT_G_CHEBYSHEV, args.g_cheb)
    if args.g_cg:
        pr.parareal_set_option(ctx, pr.PR_OPT_G_CG, args.g_cg)


def mixed_vs_fp64(pr, torch, p, u0, lam_mixed, t_mixed_ms, args, local):
    """The same solve with FP64 fine steps (same coarse solver and options), and
    the accuracy of both against the FP64 serial fine solution:
    err = max_i ||lam_i - lam*_i||_inf / max_i ||lam*_i||_inf.  The FP64 solve
    is timed on min(steps, 2) solves after one warm-up (it is the slower arm)."""
    stream = torch.cuda.current_stream()
    ctx = pr.parareal_create(local, stream)
    try:
        prob = problem_struct(pr, p, u0, None, f_prec=64)
        pr.parareal_set_problem(ctx, prob)
        apply_coarse_options(pr, ctx, args)
        lam64 = torch.empty_like(lam_mixed)
        pr.parareal_run_sync(ctx, lam64)
        n64 = max(1, min(args.steps, 2))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(n64):
            _, st = pr.parareal_run_sync(ctx, lam64)
        ev1.record(stream)
        torch.cuda.synchronize()
        t64 = ev0.elapsed_time(ev1) / n64
        star = torch.empty_like(lam_mixed)
        sst = pr.parareal_serial_fine(ctx, star)
        scale = star.abs().max().item()
        err_m = (lam_mixed - star).abs().max().item() / scale
        err_64 = (lam64 - star).abs().max().item() / scale
        return {"t_mixed_ms": t_mixed_ms, "t_fp64_ms": t64, "speedup": t64 / t_mixed_ms,
                "fp64_solves_timed": n64,
                "err_mixed": err_m, "err_fp64": err_64, "k_fp64": st.iterations,
                "fp64_t_fine_ms": st.t_fine_ms, "fp64_t_coarse_ms": st.t_coarse_ms,
                "fp64_cg_iterations": st.cg_iterations, "g_rtol": p["g_rtol"],
                "serial_fine_fp64_ms": sst.t_total_ms,
                "accuracy_target": 1e-5, "mixed_meets_target": err_m <= 1e-5}
    finally:
        pr.parareal_destroy(ctx)


def _timed(torch, fn, steps):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        res.append(fn())
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps, res


def run_async_workload(args, local):
    """Asynchronous persistent kernel vs the synchronous driver on one problem."""
    import numpy as np
    import torch

    import paper_2110_10762_gb300 as pr
    from synthetic import delay_table

    torch.cuda.set_device(local)
    p = problem_of(args.workload)
    N, M = p["N"], int(np.prod(p["n"]))
    u0 = torch.from_numpy(p["u0"].reshape(-1).copy()).cuda()
    kappa = (torch.from_numpy(p["kappa"].reshape(-1).copy()).cuda()
             if p.get("kappa") is not None else None)
    ctx = pr.parareal_create(local, torch.cuda.current_stream())
    pr.parareal_set_problem(ctx, problem_struct(pr, p, u0, kappa))
    lam = torch.empty((N + 1) * M, dtype=torch.float64, device="cuda")
    delays, unit_ns = None, 0.0
    if "delay_seed" in p:
        # one delay unit = the measured duration of one fine step of one slice
        x = lam[:M].clone()
        y = torch.empty_like(x)
        pr.parareal_fine(ctx, x, y, 1)
        t_ms, _ = _timed(torch, lambda: pr.parareal_fine(ctx, x, y, 1), 3)
        unit_ns = t_ms * 1e6 / p["f_steps"]
        delays = torch.from_numpy(delay_table(N, 64, seed=p["delay_seed"])).cuda()
    opts = pr.make_async_opts(timeout_s=300.0, delays=delays, delay_unit_ns=unit_ns,
                              lazy=args.lazy, ctas_per_slice=args.ctas_per_slice,
                              verify=args.verify)
    if args.profile:
        code, st, log = pr.parareal_run_async(ctx, opts, lam, log_cap=1 << 20)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.workload, "kappa": st.iterations, "events": st.events,
                          "t_total_ms": st.t_total_ms}), flush=True)
        pr.parareal_destroy(ctx)
        return 0
    for _ in range(args.warmup):
        pr.parareal_run_async(ctx, opts, lam, log_cap=1 << 20)
    with Clocks(local) as clk:
        t_async, res = _timed(torch, lambda: pr.parareal_run_async(ctx, opts, lam, log_cap=1 << 20),
                              args.steps)
    code, st, log = res[-1]
    lam_async = lam.clone()
    for _ in range(min(args.warmup, 1)):
        pr.parareal_run_sync(ctx, lam)
    t_sync, sres = _timed(torch, lambda: pr.parareal_run_sync(ctx, lam), args.steps)
    sst = sres[-1][1]
    launches = st.launches
    # release the async/sync workspaces before the FP64 reference (the 192^3 x 256
    # workload needs most of the device for the async rings and team buffers)
    pr.parareal_destroy(ctx)
    ctx = None
    torch.cuda.synchronize()
    # accuracy of both against the FP64 serial fine solution
    ctx64 = pr.parareal_create(local, torch.cuda.current_stream())
    pr.parareal_set_problem(ctx64, problem_struct(pr, p, u0, kappa, f_prec=64))
    star = torch.empty_like(lam)
    pr.parareal_serial_fine(ctx64, star)
    pr.parareal_destroy(ctx64)
    scale = star.abs().max().item()
    lups = sum(r[1].fine_lups for r in res)
    value = lups / (t_async * args.steps / 1e3) / 1e9
    cg_ops = {2: 10.3, 3: 12.3}[p["dim"]]
    if p.get("f_scheme") == "cn":
        f_ops = (CN_OPS_PER_CG_POINT[p["dim"]] * st.fine_cg_iterations * M
                 + CN_OPS_PER_LUP[p["dim"]] * st.fine_lups)
    elif p.get("f_prec", 64) == 64:
        f_ops = st.fine_lups * fp64_ops_per_lup(p)
    else:
        f_ops = 0
    fp64_ops = st.cg_iterations * M * cg_ops + f_ops
    roof = {"bound": "alu", "kernel": "async_kernel", "unit": "Gop/s",
            "achieved": fp64_ops / (t_async / 1e3) / 1e9, "peak": NOMINAL_FP64_OPS,
            "peak_kind": "nominal FP64 pipe", "traffic": None,
            "note": "FP64-pipe work of the CG solves"
                    + (" and FP64 fine steps" if p.get("f_prec", 64) == 64 else "")
                    + " over the whole async run (predictor included)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    out = {"metric": "fine GLUP/s", "value": value, "unit": "GLUP/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_async,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32/f64" if p.get("f_prec", 64) == 32 else "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "grid": list(p["n"]), "N": N,
                      "f_steps": p["f_steps"], "tol": p["tol"],
                      "delay_unit_ns": unit_ns, "delays": delays is not None,
                      "lazy": bool(args.lazy), "ctas_per_slice": args.ctas_per_slice,
                      "verify": bool(args.verify)},
           "async": {"status": int(code), "time_to_tol_ms": t_async, "kappa": st.iterations,
                     "verify_rounds": st.verify_rounds, "residual": st.residual,
                     "events": st.events, "cg_iterations": st.cg_iterations,
                     "fine_cg_iterations": st.fine_cg_iterations,
                     "err_vs_serial_fine": (lam_async - star).abs().max().item() / scale},
           "sync": {"time_to_tol_ms": t_sync, "k": sst.iterations,
                    "cg_iterations": sst.cg_iterations,
                    "fine_cg_iterations": sst.fine_cg_iterations,
                    "err_vs_serial_fine": (lam - star).abs().max().item() / scale},
           "async_speedup_vs_sync": t_sync / t_async,
           "sync_with_same_delays_ms": (t_sync + sync_delay_ms(delay_table(N, 64, seed=p["delay_seed"]),
                                                               unit_ns, sst.iterations, N)
                                        if delays is not None else None),
           "cost_model": cost_models(log, N, t_async, p, sst.as_dict(), t_sync),
           "kappa_over_k": st.iterations / max(sst.iterations, 1),
           "roofline": roof, "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)
    return 0


def run_adjoint_workload(args, local):
    """Loss and discrete-adjoint gradient through K sync iterations (ParaRealFn)."""
    import numpy as np
    import torch

    import paper_2110_10762_gb300 as pr
    from paper_2110_10762_gb300.autograd import ParaRealFn

    torch.cuda.set_device(local)
    p = problem_of(args.workload)
    N, M, K, nf = p["N"], int(np.prod(p["n"])), p["K"], p["f_steps"]
    T = N * nf * p["dt"]
    u0 = torch.from_numpy(p["u0"].reshape(-1).copy()).cuda()
    kap = torch.from_numpy(p["kappa"].reshape(-1).copy()).cuda()
    kstar = torch.from_numpy(p["kappa_star"].reshape(-1).copy()).cuda()
    ctx = pr.parareal_create(local, torch.cuda.current_stream())
    pr.parareal_set_problem(ctx, problem_struct(pr, p, u0, kstar))
    obs = torch.empty((N + 1) * M, dtype=torch.float64, device="cuda")
    pr.parareal_serial_fine(ctx, obs)
    pr.parareal_destroy(ctx)
    u_obs = obs[N * M:].clone()
    del obs
    spec = dict(dim=p["dim"], n=p["n"], T=T, N=N, f_steps=nf, K=K, g_rtol=p["g_rtol"])

    def step():
        a = u0.clone().requires_grad_(True)
        b = kap.clone().requires_grad_(True)
        out = ParaRealFn.apply(a, b, spec)
        loss = 0.5 * ((out - u_obs) ** 2).sum()
        loss.backward()
        return loss.item(), a.grad, b.grad

    if args.profile:
        loss, _, _ = step()
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.workload, "loss": loss}), flush=True)
        return 0
    for _ in range(args.warmup):
        step()
    with Clocks(local) as clk:
        t_ms, res = _timed(torch, step, args.steps)
    loss, gu, gk = res[-1]
    fwd = sum(N - k for k in range(K)) * M * nf
    # forward + recomputed fine states (n_f - 1 per slice) + transposed steps (n_f per slice)
    lups = fwd + sum(N - k for k in range(K)) * M * (2 * nf - 1)
    out = {"metric": "fine GLUP/s", "value": lups / (t_ms / 1e3) / 1e9, "unit": "GLUP/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "grid": list(p["n"]), "N": N,
                      "f_steps": nf, "K": K},
           "loss": loss, "grad_u0_norm": gu.norm().item(), "grad_kappa_norm": gk.norm().item(),
           "gradients_per_s": 1e3 / t_ms, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)
    return 0


def run_adjoint_async_workload(args, local):
    """Gradient of L = 1/2 ||lam_N - u_obs||^2 through a logged asynchronous run."""
    import numpy as np
    import torch

    import paper_2110_10762_gb300 as pr

    torch.cuda.set_device(local)
    p = problem_of(args.workload)
    N, M, nf = p["N"], int(np.prod(p["n"])), p["f_steps"]
    u0 = torch.from_numpy(p["u0"].reshape(-1).copy()).cuda()
    kap = torch.from_numpy(p["kappa"].reshape(-1).copy()).cuda()
    kstar = torch.from_numpy(p["kappa_star"].reshape(-1).copy()).cuda()
    ctx = pr.parareal_create(local, torch.cuda.current_stream())
    pr.parareal_set_problem(ctx, problem_struct(pr, p, u0, kstar))
    obs = torch.empty((N + 1) * M, dtype=torch.float64, device="cuda")
    pr.parareal_serial_fine(ctx, obs)
    u_obs = obs[N * M:].clone()
    del obs
    # the logged forward run (async persistent kernel, tol 1e-8)
    pr.parareal_set_problem(ctx, problem_struct(pr, p, u0, kap, tol=1e-8))
    lam = torch.empty((N + 1) * M, dtype=torch.float64, device="cuda")
    code, st, log = pr.parareal_run_async(ctx, pr.make_async_opts(timeout_s=300.0), lam,
                                          log_cap=1 << 20)
    gN = lam[N * M:] - u_obs
    gu = torch.empty(M, dtype=torch.float64, device="cuda")
    gk = torch.empty(kap.numel(), dtype=torch.float64, device="cuda")
    lamN = torch.empty(M, dtype=torch.float64, device="cuda")

    def step():
        pr.parareal_adjoint_async(ctx, log, gN, gu, gk, lamN)

    for _ in range(args.warmup):
        step()
    with Clocks(local) as clk:
        t_ms, _ = _timed(torch, step, args.steps)
    ups = len(log)
    coarse = sum(1 for e in log if e.vG > e.vF)
    # replay F (n_f) + recomputed states (n_f - 1) + transposed steps (n_f) per update
    lups = ups * M * (3 * nf - 1)
    out = {"metric": "fine GLUP/s", "value": lups / (t_ms / 1e3) / 1e9, "unit": "GLUP/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "grid": list(p["n"]), "N": N,
                      "f_steps": nf},
           "forward": {"status": int(code), "kappa": st.iterations, "events": ups,
                       "coarse_updates": coarse, "t_ms": st.t_total_ms},
           "replay_vs_run_max_abs": (lamN - lam[N * M:]).abs().max().item(),
           "grad_u0_norm": gu.norm().item(), "grad_kappa_norm": gk.norm().item(),
           "gradients_per_s": 1e3 / t_ms, "clocks": clk.summary()}
    pr.parareal_destroy(ctx)
    print(json.dumps(out), flush=True)
    return 0


# FP64 instructions per point of one coarse CG iteration (constant kappa, the
# operator scaled by 1/R_x): textbook CG d DADD + d DFMA for B p plus 5 DFMA (p.q,
# x, r, r.r, p); single-reduction d + d for B r plus 6 DFMA (p, s, x, r, r.r, w.r).
CG_OPS_PER_POINT = {("textbook", 2): 9, ("textbook", 3): 11, ("single", 2): 10, ("single", 3): 12}


def fp64_peaks(pr, torch, sm_max_mhz):
    """The FP64-pipe peak two ways: derived from unit counts and clocks (152 SMs
    x 2 FP64 instructions per clock per SM x the maximum SM clock: the nominal
    1.25 TFLOP/s FP64 of this part) and measured by the library's DFMA/DADD
    throughput probe on this device."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    mhz = sm_max_mhz or 2070.0
    derived = sms * 2 * mhz * 1e6 / 1e9
    out = {"derived_gops": derived, "derived_basis": "%d SMs x 2 FP64 instr/clk x %.0f MHz" % (
        sms, mhz), "unit": "G FP64 instr/s"}
    try:
        dfma, _ = pr.parareal_probe_fp64(0, 1 << 16)
        dadd, _ = pr.parareal_probe_fp64(1, 1 << 16)
        out.update({"probe_dfma_gops": dfma / 1e9, "probe_dadd_gops": dadd / 1e9})
    except Exception as e:   # the probe is a measurement aid; the bench line stands without it
        out["probe_error"] = str(e)
    return out


# Per-point cost of the passes of the vectorised Chebyshev-preconditioned coarse CG
# (degree m >= 4, constant kappa): (HBM bytes, FP64 instructions).  Chebyshev steps
# (FP32): the first reads f with its stencil and writes y_2 (8 B), the second
# reads y_2 and f and writes y_3 (12 B), the middle ones read y_k, y_k-1, f and
# write y_k+1 (16 B), the last also reads r in FP64 for r.z (24 B, one DFMA).
# Direction pass: z (FP32) with its stencil, p, q in; p, q out (36 B; the scaled
# operator 4 (2D) or 6 (3D) FP64 instructions, p, q, p.q one each).  Solution and
# residual pass: x, p, r, q in; x, r, f out (52 B; x, r, r.r).  Per solve: the
# start pass (x0 with its stencil, b in; r, f out: 28 B; the unscaled operator 5
# or 7, b - Bx, r.r, b.b), the fused correction (x, v, w, lambda in; lambda, w
# out: 48 B; the correction's add and subtract, the increment: 3), and the first
# direction pass in place of a full one (z in; p, q out: 20 B; operator and p.q).
# FP32 <-> FP64 conversions run on the integer pipe and count as neither.
def pcg_pass_costs(dim, m):
    op = 6 if dim == 3 else 4
    it = [(8, 0), (12, 0)] + [(16, 0)] * (m - 4) + [(24, 1), (36, op + 3), (52, 3)]
    solve = [(28, op + 4), (48, 3)]
    first_dir = (20, op + 1)
    return it, solve, first_dir


def pcg_roofline(M, dim, m, cg_its, solves, t_coarse_ms, hbm_peak, peak_kind, fp64_gops):
    """Coarse-phase roofline: each pass is bound by the larger of its HBM time and
    its FP64-pipe time; the bound of the phase is the sum over its passes."""
    it, solve, first_dir = pcg_pass_costs(dim, m)

    def t_pass(c):   # seconds per point
        return max(c[0] / (hbm_peak * 1e9), c[1] / (fp64_gops * 1e9))
    t_it = sum(t_pass(c) for c in it)
    t_solve = sum(t_pass(c) for c in solve) + t_pass(first_dir) - t_pass(it[-2])
    t_bound = M * (cg_its * t_it + solves * t_solve)
    per_it_b = sum(b for b, _ in it)
    per_solve_b = sum(b for b, _ in solve) + first_dir[0] - it[-2][0]
    gbytes = M * (cg_its * per_it_b + solves * per_solve_b)
    achieved = gbytes / (t_coarse_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "peak_kind": peak_kind, "frac": achieved / hbm_peak,
            "bytes_per_point_per_iteration": per_it_b, "bytes_per_point_per_solve": per_solve_b,
            "fp64_per_point_per_iteration": sum(f for _, f in it),
            "fp64_peak_gops": fp64_gops,
            "t_bound_ms": t_bound * 1e3, "frac_of_pass_roofline": t_bound * 1e3 / t_coarse_ms,
            "pass_roofline_note": "per pass, the larger of HBM bytes / measured copy bandwidth "
                                  "and FP64 instructions / probed DFMA rate, summed over the "
                                  "passes, over the measured coarse-phase time",
            "avg_launch_ms": t_coarse_ms / max(solves, 1),
            "algorithmic_bytes_per_launch": gbytes / max(solves, 1),
            "traffic": None}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2110_10762_gb300 as pr

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = problem_of(args.workload)
    is_mixed = p.get("f_prec", 64) == 32
    dim = p["dim"]
    M = int(np.prod(p["n"]))
    N = p["N"]
    stream = torch.cuda.current_stream()
    u0 = torch.from_numpy(p["u0"].reshape(-1).copy()).cuda()
    kappa = (torch.from_numpy(p["kappa"].reshape(-1).copy()).cuda()
             if p.get("kappa") is not None else None)
    ctx = pr.parareal_create(local, stream)
    prob = problem_struct(pr, p, u0, kappa)
    pr.parareal_set_problem(ctx, prob)
    if args.pipeline:
        pr.parareal_set_option(ctx, pr.PR_OPT_PIPELINE, 1)
        pr.parareal_set_option(ctx, pr.PR_OPT_PIPELINE_CHUNKS, args.chunks)
        pr.parareal_set_option(ctx, pr.PR_OPT_CG_BLOCKS_PER_SM, args.cg_bps)
    apply_coarse_options(pr, ctx, args)
    pr.parareal_set_option(ctx, pr.PR_OPT_F_STEPS_PER_PASS, args.f_per_pass)
    lam = torch.empty((N + 1) * M, dtype=torch.float64, device="cuda")
    if args.profile:
        code, st = pr.parareal_run_sync(ctx, lam)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.workload, "iterations": st.iterations,
                          "launches": st.launches, "t_total_ms": st.t_total_ms,
                          "cg_iterations": st.cg_iterations,
                          "coarse_solves": st.coarse_solves}), flush=True)
        pr.parareal_destroy(ctx)
        return 0

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        pr.parareal_run_sync(ctx, lam)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            code, st = pr.parareal_run_sync(ctx, lam)
            stats.append(st.as_dict())
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    lups = sum(s["fine_lups"] for s in stats)
    value, sec = replica_aggregate(lups, ev0.elapsed_time(ev1) / 1e3, world, "cuda")
    value /= 1e9
    ms = sec * 1e3
    launches = sum(s["launches"] for s in stats)
    clk_sum = clk.summary()
    # Roofline of the fine step: its launches are timed by events on the
    # library's stream around every batched F.  Under the pipelined schedule the
    # fine chunks overlap the coarse sweep, so the kernel is timed on one extra
    # solve with the plain schedule (same work, same kernels).
    roof_stats = stats
    if args.pipeline:
        pr.parareal_set_option(ctx, pr.PR_OPT_PIPELINE, 0)
        _, st_plain = pr.parareal_run_sync(ctx, lam)
        roof_stats = [st_plain.as_dict()]
        pr.parareal_set_option(ctx, pr.PR_OPT_PIPELINE, 1)
    lups_r = sum(s["fine_lups"] for s in roof_stats)
    t_fine = sum(s["t_fine_ms"] for s in roof_stats)
    t_coarse = sum(s["t_coarse_ms"] for s in roof_stats)
    cg_its = sum(s["cg_iterations"] for s in roof_stats)
    # the explicit F is one launch per fine step; the 1D implicit F and the
    # trapezoidal F (one cooperative launch over the batch) one launch per batch
    fine_launches = sum(s["iterations"] for s in roof_stats) * (
        1 if p.get("f_scheme") in ("implicit", "cn") else p["f_steps"])
    is_cn = p.get("f_scheme") == "cn" and dim > 1
    b_elem = 4 if is_mixed else 8
    alg_bytes = 2 * b_elem * lups_r  # one read + one write of the state per step
    hbm_peak, peak_kind = peaks()
    fine_glups = lups_r / (t_fine / 1e3) / 1e9
    fpk = fp64_peaks(pr, torch, clk_sum.get("sm_max_mhz"))
    fp64_peak = fpk["derived_gops"]
    fp64_meas = fpk.get("probe_dfma_gops")

    def alu_roof(ops, t_ms, kernel, extra=None):
        r = {"bound": "alu", "achieved": ops / (t_ms / 1e3) / 1e9, "peak": fp64_peak,
             "unit": "G FP64 instr/s", "traffic": None, "kernel": kernel,
             "peak_kind": "derived from unit counts and clocks (" + fpk["derived_basis"] + ")"}
        r["frac"] = r["achieved"] / r["peak"]
        if fp64_meas:
            r["peak_measured"] = fp64_meas
            r["frac_of_measured"] = r["achieved"] / fp64_meas
        if extra:
            r.update(extra)
        return r

    if is_mixed:
        tma = dim == 3 and p["n"][0] % 4 == 0 and p.get("kappa") is None
        nf = p["f_steps"]
        # passes of one F: the entry (FP64 in, FP32 out: 12 B per point; on the TMA path
        # a conversion, otherwise the first step), the steps before the last one per
        # pass or, TMA-fed, two per pass (one read and one write of the FP32 state, 8 B
        # per point per pass), and the last step (FP32 in, FP64 out: 12 B)
        if nf == 1:
            passes, bytes_pt = 1, 16
        else:
            mid = nf - 1 if tma else nf - 2
            mid_passes = (mid // 2 + mid % 2) if (tma and args.f_per_pass == 2) else mid
            passes, bytes_pt = 2 + mid_passes, 24 + 8 * mid_passes
        fine_launches = sum(s["iterations"] for s in roof_stats) * passes
        alg_bytes = bytes_pt * lups_r / nf
        roof = {"bound": "hbm", "achieved": alg_bytes / (t_fine / 1e3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "traffic": None,
                "kernel": (("step3d_tma2 (two TMA-fed FP32 steps per pass" if args.f_per_pass == 2
                            else "step3d_tma (TMA-fed FP32 steps") +
                           "; FP64 input converted by a streaming copy, last step step3d_v4 with "
                           "FP64 output)" if tma else "step3d_v4<float>"),
                "peak_kind": peak_kind,
                "bytes_per_lup": bytes_pt / nf, "passes_per_F": passes}
        roof["frac"] = roof["achieved"] / roof["peak"]
    elif is_cn:
        f_its = sum(s["fine_cg_iterations"] for s in roof_stats)
        ops = CN_OPS_PER_CG_POINT[dim] * f_its * M + CN_OPS_PER_LUP[dim] * lups_r
        roof = alu_roof(ops, t_fine, "cn_kernel (team CG per trapezoidal step)",
                        {"fine_cg_iterations_per_step": f_its / max(lups_r / M, 1)})
    else:
        ops = fp64_ops_per_lup(p) * lups_r
        # algorithmic flops of one explicit update u - dt A u: 2d + 2 (6 for the
        # 5-point stencil, 8 for the 7-point one); an FMA counts 2 against the peak
        fpl = 2 * dim + 2 if p.get("f_scheme", "explicit") == "explicit" else None
        flop_view = None
        if fpl:
            af = fpl * lups_r / (t_fine / 1e3) / 1e9
            flop_view = {"flops_per_lup": fpl, "achieved_gflops": af,
                         "peak_gflops": 2 * fp64_peak, "frac": af / (2 * fp64_peak)}
        roof = alu_roof(ops, t_fine, ("tri_solve (partition Thomas/PCR)" if dim == 1
                                      else f"step{2 if dim == 2 else 3}d<double>"),
                        {"fp64_instr_per_lup": fp64_ops_per_lup(p), "flop_view": flop_view,
                         "hbm_view": {"achieved_gbs": alg_bytes / (t_fine / 1e3) / 1e9,
                                      "peak_gbs": hbm_peak,
                                      "frac": alg_bytes / (t_fine / 1e3) / 1e9 / hbm_peak}})
    roof["avg_launch_ms"] = t_fine / max(fine_launches, 1)
    lups_per_launch = lups_r / max(fine_launches, 1)
    tpl = NCU_TRAFFIC_PER_LUP.get(args.workload)
    if is_mixed:
        # per launch of the dominant kernel (a middle pass over the active slices):
        # the algorithmic bytes and the ncu DRAM bytes scaled to the same points
        steps_per_pass = 2 if (roof.get("passes_per_F", 0) < p["f_steps"]) else 1
        pts = lups_r / p["f_steps"] / max(sum(s["iterations"] for s in roof_stats), 1)
        roof["algorithmic_bytes_per_launch"] = 8.0 * pts
        roof["traffic"] = (tpl * steps_per_pass * pts
                           if tpl and steps_per_pass == 2 and args.f_per_pass == 2 else None)
        roof["note"] = ("achieved = algorithmic bytes of all passes of the F phase (first and last "
                        "with FP64 I/O) / F-phase time; per-launch figures are for a middle pass")
    else:
        roof["algorithmic_bytes_per_launch"] = 2 * b_elem * lups_per_launch
        roof["traffic"] = tpl * lups_per_launch if tpl else None
    # coarse sweep (the predictor and the corrections' CG solves): FP64 pipe
    roof_coarse = None
    if p.get("g_solver") != "thomas" and not args.g_cheb and p.get("kappa") is None:
        rec = "single" if args.g_cg == 2 else "textbook"
        ops_g = CG_OPS_PER_POINT[(rec, dim)] * cg_its * M
        roof_coarse = alu_roof(ops_g, t_coarse, "cg_kernel (%s CG recurrence)" % rec,
                               {"cg_iterations": cg_its,
                                "us_per_cg_iteration": t_coarse * 1e3 / max(cg_its, 1),
                                "note": "coarse-phase time includes each solve's start and "
                                        "fused-correction passes"})
    elif p.get("g_solver") != "thomas":
        roof_coarse = {"kernel": "cg_kernel (Chebyshev-preconditioned CG, %d FP32 steps)" % args.g_cheb
                       if args.g_cheb else "cg_kernel",
                       "cg_iterations": cg_its,
                       "us_per_cg_iteration": t_coarse * 1e3 / max(cg_its, 1)}
        vec = dim >= 2 and p.get("kappa") is None and p["n"][0] % 4 == 0
        if args.g_cheb >= 4 and vec:
            roof_coarse.update(pcg_roofline(M, dim, args.g_cheb, cg_its,
                                            sum(s["coarse_solves"] for s in roof_stats),
                                            t_coarse, hbm_peak, peak_kind,
                                            fpk.get("probe_dfma_gops") or fp64_peak))
            ratio = NCU_COARSE_TRAFFIC_RATIO.get(args.workload)
            if ratio:
                roof_coarse["traffic"] = ratio * roof_coarse["algorithmic_bytes_per_launch"]
    # the bench line's roofline is that of the kernel with the larger share of the solve
    dominant = roof
    if roof_coarse and roof_coarse.get("frac") is not None and t_coarse > t_fine:
        dominant = dict(roof_coarse, share_of_solve=t_coarse / (t_fine + t_coarse))
    else:
        dominant = dict(roof, share_of_solve=t_fine / max(t_fine + t_coarse, 1e-9))
    out = {"metric": "fine GLUP/s", "value": value, "unit": "GLUP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32/f64" if is_mixed else "f64", "data": "synthetic",
           "config": bench_config(args, p, world),
           "iterations": stats[-1]["iterations"], "time_to_tol_ms": ms / args.steps,
           "fine_phase_glups": fine_glups,
           "t_fine_ms_per_solve": t_fine / len(roof_stats),
           "t_coarse_ms_per_solve": t_coarse / len(roof_stats),
           "cg_iterations_per_step": sum(s["cg_iterations"] for s in stats) / args.steps,
           "predictor": {"cg_iterations": roof_stats[-1]["predictor_cg_iterations"],
                         "t_ms": roof_stats[-1]["t_predictor_ms"]},
           "cost_model": cost_model_sync(p, roof_stats[-1], roof_stats[-1]["t_total_ms"]),
           "roofline": dominant, "roofline_fine": roof, "roofline_coarse": roof_coarse,
           "fp64_peak": fpk,
           "gpu_launches": launches}
    # GPU serial fine solve on the same problem (time-to-solution reference)
    sf = torch.empty_like(lam)
    sst = pr.parareal_serial_fine(ctx, sf)
    sst = pr.parareal_serial_fine(ctx, sf)
    out["serial_fine_gpu_ms"] = sst.t_total_ms
    out["speedup_vs_gpu_serial_fine"] = sst.t_total_ms / (ms / args.steps)
    diff = (lam - sf).abs().max().item()
    out["max_abs_vs_serial_fine"] = diff
    del sf
    if is_mixed and not args.no_fp64:
        mv = mixed_vs_fp64(pr, torch, p, u0, lam, ms / args.steps, args, local)
        mv["serial_fine_fp32_ms"] = sst.t_total_ms
        out["mixed_vs_fp64"] = mv
        out["speedup_vs_gpu_serial_fine_fp64"] = mv["serial_fine_fp64_ms"] / (ms / args.steps)
    # end-to-end through the host-buffer entry point (pinned host memory); long
    # solves are timed on at most three of them
    if not args.no_e2e:
        e_steps = args.steps if ms / args.steps < 3000 else max(1, min(args.steps, 3))
        u0h = torch.from_numpy(p["u0"].reshape(-1).copy()).pin_memory()
        outh = torch.empty((N + 1) * M, dtype=torch.float64).pin_memory()
        pr.parareal_run_sync_host(ctx, u0h, outh)
        barrier()
        with Clocks(local) as clk_e:
            t0 = time.perf_counter()
            e_lups = 0
            for _ in range(e_steps):
                _, st = pr.parareal_run_sync_host(ctx, u0h, outh)
                e_lups += st.fine_lups
            torch.cuda.synchronize()
            e_sec = time.perf_counter() - t0
        e_value, _ = replica_aggregate(e_lups, e_sec, world, "cuda")
        out["e2e"] = {"value": e_value / 1e9, "unit": "GLUP/s",
                      "h2d_bytes_per_step": M * 8, "d2h_bytes_per_step": (N + 1) * M * 8,
                      "steps": e_steps, "ms_per_step": e_sec * 1e3 / e_steps,
                      "clocks": clk_e.summary()}
        del outh
    out["clocks"] = clk_sum
    stats_last = dict(roof_stats[-1])
    pr.parareal_destroy(ctx)
    if rank == 0 and not args.no_cpu:
        base, over = preset_args(args.workload)
        out["cpu_baseline"] = cpu_baseline_leg(base, p, over, stats_last)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    global G_RTOL_OVERRIDE
    args = parse()
    G_RTOL_OVERRIDE = args.g_rtol
    if args.grid:
        SIZE_OVERRIDE["n"] = tuple(int(v) for v in args.grid.split(","))
    if args.slices:
        SIZE_OVERRIDE["N"] = args.slices
    if args.g_cheb is None:
        from synthetic.configs import PRESETS
        args.g_cheb = int(PRESETS[preset_args(args.workload)[0]].get("g_cheb", 0))
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload in ("heat2d_async", "heat3d_varkappa_async", "heat2d_cn_async"):
        return run_async_workload(args, local) if rank == 0 else 0
    if args.workload == "heat2d_inverse_async":
        return run_adjoint_async_workload(args, local) if rank == 0 else 0
    if args.workload == "heat2d_inverse":
        return run_adjoint_workload(args, local) if rank == 0 else 0
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
