#!/usr/bin/env python
"""Benchmark: synchronous Parareal on the 2D heat workload, one JSON line.

Workload (default "heat2d_explicit"): u_t = Laplace(u) on the unit square,
1024 x 1024 interior grid, zero Dirichlet boundary, N = 64 slices, F = 256
explicit-Euler 5-point steps per slice at dt = 0.2 h^2, G = one implicit
Euler step per slice solved by CG (rtol 1e-10), u0 = 32 random sine modes +
8 Gaussian bumps (seeded), FP64, stop when max_i ||lam_i^k - lam_i^{k-1}||_inf
< 1e-10.  One "step" = one complete Parareal solve (predictor, batched fine
sweeps, coarse sweeps with the fused correction and test) to the tolerance.

metric: fine GLUP/s = fine cell updates executed / wall time of the solves.

Multi-GPU (torchrun): replicas only -- every rank solves its own copy of the
workload; value = units of all ranks / max-over-ranks time (weak scaling).
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "heat2d_explicit": "2D heat 1024x1024, N=64 slices, F=256 explicit 5-pt steps (dt=0.2h^2), "
                       "G=1 implicit Euler step by CG (rtol 1e-10), FP64, sync Parareal, tol 1e-10",
    "heat3d_mixed": "3D heat 256^3, N=128 slices, F=64 explicit 7-pt steps (dt=0.15h^2), "
                    "G=implicit Euler by CG (rtol 1e-10), FP32 fine / FP64 coarse, sync, tol 1e-5",
}
# FP64-pipe operations per fine cell update of the explicit step (DADD/DMUL/DFMA
# each one issue slot): 2D 5-point = 2 DADD + 1 DMUL + 2 DFMA; 3D 7-point = 3 + 1 + 3.
FP64_OPS_PER_LUP = {2: 5, 3: 7}
NOMINAL_FP64_OPS = 625.0  # G FP64-pipe ops/s: 1.25 TFLOP/s nominal / 2 flops per DFMA


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heat2d_explicit", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
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


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def problem_of(name):
    from synthetic import preset
    p = preset(name, "full")
    return p


def cpu_sample(p, slices=2, steps=None):
    """The FP64 oracle's fine propagator on a bounded sample of the workload."""
    import numpy as np
    from oracle import heat
    steps = p["f_steps"] if steps is None else steps
    P = heat.Propagators(dict(p, f_steps=steps))
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    for _ in range(slices):
        P.F(p["u0"] + 0.01 * rng.standard_normal(p["u0"].shape))
    dt = time.perf_counter() - t0
    lups = slices * steps * int(np.prod(p["n"]))
    return lups / dt / 1e9, dt, lups


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    p = problem_of(args.workload)
    steps_per_sample = 64 if p["dim"] == 2 else 4
    for _ in range(args.warmup):
        cpu_sample(p, 1, steps_per_sample)
    tot_t, tot_l = 0.0, 0
    for _ in range(args.steps):
        _, dt, l = cpu_sample(p, 1, steps_per_sample)
        tot_t += dt
        tot_l += l
    v = tot_l / tot_t / 1e9
    sample = (f"oracle F (numpy FP64) on 1 slice x {steps_per_sample} fine steps of the "
              f"full {'x'.join(map(str, p['n']))} grid per step")
    out = {"impl": "reference", "metric": "fine GLUP/s", "value": v, "unit": "GLUP/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload]},
           "cpu_baseline": {"value": v, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


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
    ctx = pr.parareal_create(local, stream)
    prob = pr.make_problem(dim=dim, n=p["n"], T0=0.0, T=N * p["f_steps"] * p["dt"], N=N, u0=u0,
                           f_steps=p["f_steps"], f_prec=p.get("f_prec", 64),
                           g_rtol=p["g_rtol"], tol=p["tol"])
    pr.parareal_set_problem(ctx, prob)
    lam = torch.empty((N + 1) * M, dtype=torch.float64, device="cuda")

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
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    lups = sum(s["fine_lups"] for s in stats)
    value = lups * world / (ms / 1e3) / 1e9
    t_fine = sum(s["t_fine_ms"] for s in stats)
    launches = sum(s["launches"] for s in stats)
    fine_launches = sum(s["iterations"] for s in stats) * p["f_steps"]
    # dominant kernel: the explicit fine step (its launches, timed by events on the
    # library's stream around every batched F)
    b_elem = 4 if is_mixed else 8
    alg_bytes = 2 * b_elem * lups  # one read + one write of the state per step
    hbm_peak, peak_kind = peaks()
    fine_glups = lups / (t_fine / 1e3) / 1e9
    if is_mixed:
        roof = {"bound": "hbm", "achieved": alg_bytes / (t_fine / 1e3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "traffic": None, "kernel": "step3d<float>",
                "peak_kind": peak_kind}
    else:
        ops = FP64_OPS_PER_LUP[dim] * lups
        roof = {"bound": "alu", "achieved": ops / (t_fine / 1e3) / 1e9, "peak": NOMINAL_FP64_OPS,
                "unit": "Gop/s", "traffic": None,
                "kernel": f"step{2 if dim == 2 else 3}d<double>",
                "peak_kind": "nominal FP64 (1.25 TFLOP/s = 625 G DFMA/s)",
                "hbm_view": {"achieved_gbs": alg_bytes / (t_fine / 1e3) / 1e9, "peak_gbs": hbm_peak,
                             "frac": alg_bytes / (t_fine / 1e3) / 1e9 / hbm_peak}}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["avg_launch_ms"] = t_fine / max(fine_launches, 1)
    out = {"metric": "fine GLUP/s", "value": value, "unit": "GLUP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32/f64" if is_mixed else "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "grid": list(p["n"]), "N": N,
                      "f_steps": p["f_steps"], "tol": p["tol"],
                      "parallelism": "replicas" if world > 1 else "1 GPU",
                      "l2": "inputs larger than L2 (trajectory %.2f GB + workspaces)" % (
                          (N + 1) * M * 8 / 1e9)},
           "iterations": stats[-1]["iterations"], "time_to_tol_ms": ms / args.steps,
           "fine_phase_glups": fine_glups,
           "t_fine_ms_per_step": t_fine / args.steps,
           "t_coarse_ms_per_step": sum(s["t_coarse_ms"] for s in stats) / args.steps,
           "cg_iterations_per_step": sum(s["cg_iterations"] for s in stats) / args.steps,
           "roofline": roof, "gpu_launches": launches}
    # GPU serial fine solve on the same problem (time-to-solution reference)
    sf = torch.empty_like(lam)
    sst = pr.parareal_serial_fine(ctx, sf)
    sst = pr.parareal_serial_fine(ctx, sf)
    out["serial_fine_gpu_ms"] = sst.t_total_ms
    out["speedup_vs_gpu_serial_fine"] = sst.t_total_ms / (ms / args.steps)
    diff = (lam - sf).abs().max().item()
    out["max_abs_vs_serial_fine"] = diff
    del sf
    # end-to-end through the host-buffer entry point (pinned host memory)
    if not args.no_e2e:
        u0h = torch.from_numpy(p["u0"].reshape(-1).copy()).pin_memory()
        outh = torch.empty((N + 1) * M, dtype=torch.float64).pin_memory()
        pr.parareal_run_sync_host(ctx, u0h, outh)
        barrier()
        t0 = time.perf_counter()
        e_lups = 0
        for _ in range(args.steps):
            _, st = pr.parareal_run_sync_host(ctx, u0h, outh)
            e_lups += st.fine_lups
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([te], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        out["e2e"] = {"value": e_lups * world / te / 1e9, "unit": "GLUP/s",
                      "h2d_bytes_per_step": M * 8, "d2h_bytes_per_step": (N + 1) * M * 8}
    out["clocks"] = clk.summary()
    pr.parareal_destroy(ctx)
    if rank == 0 and not args.no_cpu:
        v, dt, l = cpu_sample(p, slices=2 if dim == 2 else 1, steps=None if dim == 2 else 4)
        out["cpu_baseline"] = {"value": v, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                               "sample": "oracle F (numpy FP64, single thread) on %s fine "
                                         "steps of the full grid, %.1f s" % (
                                             "2 slices x %d" % p["f_steps"] if dim == 2
                                             else "1 slice x 4", dt)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
