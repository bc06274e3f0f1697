#!/usr/bin/env python3
"""Benchmark of the matrix-free monolithic multigrid Stokes solver on one GB300 (or N replicas).

Workload (one "step"): three solves of the 3D generalized Stokes system, Q2-Q1 Taylor-Hood on
32^3 hexahedra of the unit cube whose vertices are moved by a smooth seeded field of amplitude
0.1 h (trilinear cells), 5 levels, mu = rho = 1, gamma in {0, 1e2, 1e4}; right-hand side
b = M_v f with a 4-mode Fourier forcing (seed 0); FP64 flexible GMRES(30) right-preconditioned
by one FP32 V-cycle (Chebyshev degrees k_A = k_S = 3, m = 2) to ||b - K x|| <= 1e-8 ||b||,
from x = 0.  Setup (hierarchy, diagonals, Lanczos, coarse inverse) is outside the timed region.

Metric: MDoF/s solved (DoFs per second of time-to-1e-8; the inverse of solve time per MDoF),
with FP64-MG, vmult throughput, roofline of the dominant kernel, end-to-end throughput through
the host-buffer C call, and the CPU oracle baseline reported beside it.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MDoF/s Stokes vmult; solve time/MDoF to 1e-8 residual, FP32-MG vs FP64-MG"
WL = dict(dim=3, k=2, n=(32, 32, 32), levels=5, amplitude=0.1, seed=0, gammas=(0.0, 1e2, 1e4), rtol=1e-8,
          kA=3, kS=3, m=2, restart=30)
WORKLOAD_NAME = ("3D generalized Stokes Q2-Q1, unit cube 32^3 hexes, smooth trilinear vertex perturbation "
                 "0.1h (seed 0), 5 levels, mu=rho=1, gamma in {0,1e2,1e4}, FGMRES(30)+FP32 V-cycle "
                 "(kA=kS=3, m=2), rtol 1e-8")
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0


def dofs(n, k=2, dim=3):
    nu = dim
    npr = 1
    for a in range(dim):
        nu *= k * n[a] + 1
        npr *= (k - 1) * n[a] + 1
    return nu + npr


def flops_per_cell_A(k, trilinear, dim=3):
    """Algorithmic flops of one cell of the velocity-block apply (A u) by sum factorisation.

    Per component: forward interpolation d sweeps and collocation gradient d sweeps, backward
    the transposes (4 d (k+1)^d (k+1) multiply-adds), the point operation (d^2 multiply-adds
    plus 5 flops per point).  Trilinear geometry (3D, as the column kernel evaluates it): per
    (x, y) node column 78 flops to set up the edge vectors of the Jacobian, per point 83 flops
    (two Jacobian columns linear in zeta, adjugate, determinant, w/det, G = w adj adj^T / det,
    w det).  Cartesian cells: geometry is a constant.
    """
    n1 = k + 1
    npt = n1 ** dim
    per_comp = 2 * (4 * dim * npt * n1 + dim * dim * npt) + 5 * npt
    geo = 0
    if trilinear:
        geo = n1 ** (dim - 1) * 78 + npt * 83
    return dim * per_comp + geo


def fp32_peak_tflops(sm_count, clock_mhz):
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count * 128 * 2 * clock_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------------------------
def perturbed_vertices():
    import workloads as W
    return W.perturbed_vertices(WL["dim"], WL["n"], seed=WL["seed"], amplitude=WL["amplitude"])


def forcing():
    import workloads as W
    return W.fourier_forcing(WL["dim"], WL["k"], WL["n"], seed=WL["seed"]).reshape(-1)


def oracle_sample(steps=1, warmup=0):
    """CPU oracle on a bounded sample of the workload: the 16^3 level of the same perturbed
    hierarchy (every second vertex of the 32^3 mesh; 112,724 DoFs, 4 levels), the same three
    gamma values, FP64 multigrid + FGMRES to 1e-8.  Returns seconds per step (3 solves)."""
    import numpy as np
    from oracle.assemble import load_vector_nodal
    from oracle.krylov import fgmres
    from oracle.mesh import Hierarchy
    from oracle.mg import Multigrid
    import workloads as W
    V = perturbed_vertices()[::2, ::2, ::2]
    n = tuple(c // 2 for c in WL["n"])
    H = Hierarchy(3, 2, n, WL["levels"] - 1, V)
    lev = H.levels[-1]
    f = W.fourier_forcing(3, 2, n, seed=WL["seed"]).reshape(-1)
    mgs, bs = [], []
    for g in WL["gammas"]:
        mg = Multigrid(H, gamma_rho=g, kA=WL["kA"], kS=WL["kS"], m=WL["m"])
        mgs.append(mg)
        bs.append(load_vector_nodal(lev, mg.ops[-1], f))
    times, iters = [], []
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        its = []
        for mg, b in zip(mgs, bs):
            _, it, _ = fgmres(lambda v, mg=mg: mg.K @ v, mg.precondition, b, rtol=WL["rtol"], restart=WL["restart"])
            its.append(it)
        dt = time.perf_counter() - t0
        if s >= warmup:
            times.append(dt)
            iters = its
    return {"seconds_per_step": sum(times) / len(times), "dofs": lev.size, "solves_per_step": len(WL["gammas"]),
            "iterations": iters, "steps": steps}


def run_oracle_subprocess(steps=1, warmup=0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--_oracle-sample", str(steps), str(warmup)],
                       capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return None, "fallback"


def traffic_record(kernel_src_sha):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p))
    except Exception:
        return None
    if rec.get("kernel_source_sha256") != kernel_src_sha:
        return None
    return rec.get("dram_bytes_per_launch_full_size")


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("apply.cuh", "apply_col.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2205_15770_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


# ---------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2205_15770_gb300 import StokesMG

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier(device_ids=[local])

    V = perturbed_vertices()
    N = dofs(WL["n"])
    f = torch.as_tensor(forcing(), device="cuda")
    common = dict(dim=3, n=WL["n"], n_levels=WL["levels"], k=WL["k"], vertices=V, kA=WL["kA"], kS=WL["kS"],
                  m=WL["m"], restart=WL["restart"])
    t0 = time.perf_counter()
    S32 = [StokesMG(gamma_rho=g, vcycle_fp32=True, **common) for g in WL["gammas"]]
    setup_s = (time.perf_counter() - t0) / len(S32)
    S64 = [StokesMG(gamma_rho=g, vcycle_fp32=False, **common) for g in WL["gammas"]]
    B = [S.mass_rhs(f) for S in S32]
    X = [torch.zeros(N, dtype=torch.float64, device="cuda") for _ in S32]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(solvers, xs):
        its = []
        for S, b, x in zip(solvers, B, xs):
            x.zero_()
            _, it, rel = S.solve(b, x, rtol=WL["rtol"])
            its.append(it)
        return its

    for _ in range(args.warmup):
        step(S32, X)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if args.profile_range:
        torch.cuda.profiler.start()
    l0 = sum(S.launch_count for S in S32)
    total_ms = 0.0
    iters = None
    for _ in range(args.steps):
        flush.zero_()  # L2 flush (256 MB write) between timed steps, outside the events
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        iters = step(S32, X)
        e1.record()
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    launches = sum(S.launch_count for S in S32) - l0
    if args.profile_range:
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    barrier()
    t_max = total_ms
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    ms_per_step = t_max / args.steps
    solves = len(WL["gammas"])
    value = world * solves * N / (ms_per_step / 1e3) / 1e6

    # --- final residuals of the timed solves (FP64 operator on the GPU) ------------------------
    rels = []
    for S, b, x in zip(S32, B, X):
        r = b - S.vmult(x)
        rels.append(float(torch.linalg.norm(r) / torch.linalg.norm(b)))

    # --- FP64-MG comparison (same solves, FP64 V-cycle) -----------------------------------------
    X64 = [torch.zeros_like(x) for x in X]
    step(S64, X64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record()
    it64 = step(S64, X64)
    e1.record()
    e1.synchronize()
    ms64 = e0.elapsed_time(e1)
    diff = max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(X, X64))

    # --- vmult throughput ----------------------------------------------------------------------
    vm = {}
    for prec, dt in ((32, torch.float32), (64, torch.float64)):
        xv = torch.randn(N, dtype=dt, device="cuda")
        yv = torch.empty_like(xv)
        S = S32[1]
        for _ in range(3):
            S.vmult(xv, yv)
        reps = 50 if prec == 32 else 10
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            S.vmult(xv, yv)
        e1.record()
        e1.synchronize()
        vm[f"fp{prec}"] = N / (e0.elapsed_time(e1) / reps / 1e3) / 1e6

    # --- roofline of the dominant kernel (velocity-block cell apply, FP32, finest level) --------
    S = S32[1]
    S.time_apply(1, precision=32, reps=20)
    avg_ms = S.time_apply(1, precision=32, reps=200)
    n_cells = WL["n"][0] * WL["n"][1] * WL["n"][2]
    fl = flops_per_cell_A(WL["k"], True) * n_cells
    achieved = fl / (avg_ms / 1e3) / 1e12
    props = torch.cuda.get_device_properties(local)
    max_mhz = clk["sm_max_mhz"] if clk else 2070.0
    peak = fp32_peak_tflops(props.multi_processor_count, max_mhz)
    traffic = traffic_record(kernel_source_sha())
    avg64 = S.time_apply(1, precision=64, reps=10)

    # --- end to end through the host-buffer C call ----------------------------------------------
    bh = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in S32]
    xh = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in S32]
    for t, b in zip(bh, B):
        t.copy_(b.cpu())
    bn = [t.numpy() for t in bh]
    xn = [t.numpy() for t in xh]
    for S, b, x in zip(S32, bn, xn):
        S.solve_host(b, rtol=WL["rtol"], out=x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for S, b, x in zip(S32, bn, xn):
            S.solve_host(b, rtol=WL["rtol"], out=x)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_val = world * solves * N / e2e_s / 1e6

    peaks, peaks_src = measured_peaks()
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "MDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "dofs_per_solve": N, "solves_per_step": solves,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "flushed by a 256 MB write before every timed step"},
        "iterations_fp32_mg": iters, "final_rel_residual": rels,
        "solve_ms": {"fp32_mg_per_solve": round(ms_per_step / solves, 3), "fp64_mg_per_solve": round(ms64 / solves, 3)},
        "solve_s_per_mdof": {"fp32_mg": ms_per_step / solves / 1e3 / (N / 1e6),
                             "fp64_mg": ms64 / solves / 1e3 / (N / 1e6)},
        "iterations_fp64_mg": it64, "fp32_vs_fp64_mg_solution_rel_diff": diff,
        "vmult_mdof_s": {k2: round(v, 1) for k2, v in vm.items()},
        "setup_s_per_context": round(setup_s, 3),
        "roofline": {"bound": "alu", "kernel": "stokes_cell_apply<3,2,float,trilinear> (A block)",
                     "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "avg_launch_us": round(avg_ms * 1e3, 2), "flops_per_launch": fl,
                     "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                     "fp64_avg_launch_us": round(avg64 * 1e3, 2),
                     "hbm_peak_gbs": (peaks or {}).get("hbm_gbs", FALLBACK_HBM_GBS),
                     "hbm_peak_source": peaks_src},
        "e2e": {"value": round(e2e_val, 3), "unit": "MDoF/s", "h2d_bytes_per_step": solves * N * 8,
                "d2h_bytes_per_step": solves * N * 8},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            o = run_oracle_subprocess(1, 0)
            out["cpu_baseline"] = {"value": round(o["solves_per_step"] * o["dofs"] / o["seconds_per_step"] / 1e6, 4),
                                   "unit": "MDoF/s", "cores": 1, "kind": "oracle",
                                   "sample": ("3 FP64-MG FGMRES solves to 1e-8 (gamma 0, 1e2, 1e4) on the 16^3 level "
                                              "of the same perturbed hierarchy (112,724 DoFs, 4 levels), "
                                              "numpy/scipy, 1 thread; setup untimed"),
                                   "iterations": o["iterations"]}
        except Exception as e:  # report, do not hide
            out["cpu_baseline"] = {"value": None, "error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(out))
    for S in S32 + S64:
        S.close()
    if world > 1:
        dist.destroy_process_group()


def run_kernel_only(args):
    """Set up one FP32 context of the workload (gamma = 1e2) and launch the dominant kernel (A-block
    cell apply, FP32, finest level) a few times inside a cudaProfilerStart/Stop range; for ncu."""
    import torch
    from paper_2205_15770_gb300 import StokesMG
    torch.cuda.set_device(0)
    S = StokesMG(dim=3, n=WL["n"], n_levels=WL["levels"], k=WL["k"], vertices=perturbed_vertices(), gamma_rho=1e2,
                 kA=WL["kA"], kS=WL["kS"], m=WL["m"])
    S.time_apply(1, precision=32, reps=3)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    ms = S.time_apply(1, precision=32, reps=3)
    torch.cuda.profiler.stop()
    print(json.dumps({"kernel": "stokes_cell_apply A-block fp32", "avg_launch_us": ms * 1e3,
                      "cells": WL["n"][0] * WL["n"][1] * WL["n"][2]}))
    S.close()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    o = run_oracle_subprocess(args.steps, args.warmup)
    value = o["solves_per_step"] * o["dofs"] / o["seconds_per_step"] / 1e6
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MDoF/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(o["seconds_per_step"] * 1e3, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "dofs_per_solve": o["dofs"], "solves_per_step": o["solves_per_step"],
                   "parallelism": "single"},
        "cpu_baseline": {"value": round(value, 4), "unit": "MDoF/s", "cores": 1, "kind": "oracle",
                         "sample": ("each step: 3 FP64-MG FGMRES solves to 1e-8 (gamma 0, 1e2, 1e4) on the 16^3 "
                                    "level of the same perturbed hierarchy (112,724 DoFs), numpy/scipy, 1 thread")},
        "e2e": {"value": round(value, 4), "unit": "MDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "iterations": o["iterations"],
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps by cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only launch the dominant kernel inside a profiler range (for ncu --set full)")
    ap.add_argument("--_oracle-sample", nargs=2, type=int, default=None, dest="oracle_sample")
    args = ap.parse_args()
    if args.oracle_sample is not None:
        print(json.dumps(oracle_sample(*args.oracle_sample)))
        return
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.kernel_only:
        run_kernel_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
