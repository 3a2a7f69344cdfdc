#!/usr/bin/env python
"""Benchmark of the LDU pressure solve on one GB300 (replicas on N GPUs).

Workload (the 8M-cell configuration the metric is quoted on): a 200^3 hex
block, interior points jittered by U(-0.2, 0.2) h, cells randomly permuted,
faces re-sorted to upper-triangular order, face diffusivity log-normal
(sigma = 1), Dirichlet p = 0 on x-max, b ~ N(0, 1), seed 3; DIC
preconditioning, tolerance 1e-8 (normalised residual).

One step = laplacian assembly from the resident geometry + the mixed-precision
solve (FP32 DIC-PCG inside FP64 refinement) to 1e-8.  The FP64 solve of the
same system and the stand-alone Amul are timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time to 1e-8 rel. residual @8M cells (FP64 vs mixed); Amul HBM GB/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the mixed-precision solve kernel, from a one-kernel, one-launch ncu capture
# of the 128^3 case (seed 2 recipe) with its iteration counts; scaled to the
# bench workload by the per-iteration byte model (traffic grows with the
# algorithmic bytes).  Valid only for the solver source it was taken with
# (checked by hash, else the line reports null).
TRAFFIC = {"solve_cu_sha1": "b6798d6b171cc9be79cdaa9c0490dba6469f33d1", "n": 128,
           "bytes": 124937681920 + 2498494208, "inner": 524, "outer": 4}
# Iteration counts of this seeded workload (mixed: inner iterations, outer
# steps), used only to project the CPU oracle's bounded sample to a full solve.
PROJECTION_ITERS = {"inner": 795, "outer": 5}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=200, help="mesh side (default 200: 8.0M cells)")
    ap.add_argument("--cpu-iters", type=int, default=24, help="oracle inner iterations in the CPU sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", action="store_true",
                    help="time the batched workload instead: 64 systems, cells log-uniform in 1e4..5e5")
    ap.add_argument("--profile-run", action="store_true",
                    help="one launch of each hot kernel on the n^3 workload (for profiler captures): no timing")
    ap.add_argument("--seed", type=int, default=None, help="workload seed (default 3 at 200^3, else 2)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def traffic_bytes(n_cells: int, n_faces: int, inner: int, outer: int):
    """The recorded DRAM traffic of one solve launch, scaled from the captured
    case to this one by the algorithmic bytes, when the solver source still
    matches the capture; else None."""
    import hashlib
    if not TRAFFIC["bytes"]:
        return None
    src = os.path.join(ROOT, "paper_2512_22215_gb300", "csrc", "solve.cu")
    with open(src, "rb") as fh:
        sha = hashlib.sha1(fh.read()).hexdigest()
    if sha != TRAFFIC["solve_cu_sha1"]:
        return None
    n = TRAFFIC["n"]
    nf = 3 * (n - 1) * n * n
    wc, wb = workload_bytes(n ** 3, nf), workload_bytes(n_cells, n_faces)
    cap = TRAFFIC["inner"] * wc["it32"] + (TRAFFIC["outer"] + 1) * wc["resid64"]
    this = inner * wb["it32"] + (outer + 1) * wb["resid64"]
    return int(TRAFFIC["bytes"] * this / cap)


def workload_bytes(n_cells: int, n_faces: int):
    """Algorithmic bytes (LDU basis, int32 indices) of one PCG iteration and of
    one Amul: FP64 iteration 152N + 48F, FP32 iteration 76N + 36F, FP64 Amul
    16F + 24N, FP32 Amul 12F + 12N, FP64 residual b - A x 16F + 40N."""
    N, F = n_cells, n_faces
    return dict(it64=152 * N + 48 * F, it32=76 * N + 36 * F, amul64=16 * F + 24 * N, amul32=12 * F + 12 * N,
                resid64=16 * F + 40 * N)


def parse_cpulist(text: str) -> set:
    """CPU numbers of a sysfs cpulist ("0-3,8,10-11")."""
    cpus = set()
    for part in text.strip().split(","):
        if part:
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_to_gpu_cpus(index: int) -> str:
    """Restrict this process to the CPUs next to GPU `index` (the GPU's
    local_cpulist in sysfs), so that pinned host buffers are allocated in the
    GPU's NUMA node and the end-to-end copies do not cross the CPU link.
    Returns what was done, for the JSON line."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/local_cpulist"
        cpus = parse_cpulist(open(path).read()) & os.sched_getaffinity(0)
        if not cpus:
            return "unchanged (no local CPU available)"
        os.sched_setaffinity(0, cpus)
        return f"{len(cpus)} CPUs local to the GPU"
    except Exception as e:   # no sysfs entry, no nvidia-smi: keep the inherited affinity
        return f"unchanged ({type(e).__name__})"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index: int):
        # SPUMA_CLOCKS_DIR keeps the raw samples (default: the system temporary directory)
        import tempfile
        self.path = os.path.join(os.environ.get("SPUMA_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"spuma_clocks_{os.getpid()}.csv")
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_case(n: int, seed=None):
    import hexmesh
    if seed is None:
        seed = 3 if n == 200 else 2
    return hexmesh.pressure_case(n, jitter=0.2, permute=True, seed=seed, lognormal_gamma=True)


def profile_run(args, local):
    """One launch of each hot kernel on the n^3 workload, in this order: the
    assembly, a mixed solve, an FP64 solve, the pressure-step operators
    (weights, gradient, right-hand side, flux, divergence), the stand-alone
    FP64 and FP32 Amul on the prepared matrix, and a GAMG solve (two-stage
    Gauss-Seidel, algebraic pairing).  For profiler captures (-k selects the
    kernel); prints one line."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_22215_gb300 import MIXED, LduMesh, SolverControls
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = make_case(args.n, args.seed)
    m = case.mesh
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M = LduMesh(m.lower, m.upper_addr, m.n_cells, device=dev, centres=m.c)
    sf, cc, cf, v = T(m.sf), T(m.c), T(m.cf), T(m.v)
    bcell, bsf, bcf, bg, bt = T(m.bface_cell), T(m.bface_sf), T(m.bface_cf), T(case.bgamma), T(case.btype)
    gamma, b = T(case.gamma), T(case.b)
    up, dg = M.assemble_laplacian(sf, cc, gamma, bcell, bsf, bcf, bg, bt)
    _, pm = M.solve(dg, up, b, None, SolverControls(precond=2, precision=MIXED, tolerance=1e-8))
    _, pf = M.solve(dg, up, b, None, SolverControls(precond=2, tolerance=1e-8))
    rng = np.random.default_rng(7)
    phi = T(rng.standard_normal(m.n_faces) * np.linalg.norm(m.sf, axis=1))
    bphi = T(rng.standard_normal(m.n_bfaces) * np.linalg.norm(m.bface_sf, axis=1))
    w = M.fv_weights(sf, cf, cc)
    g = M.fv_grad(sf, w, v, b, bcell, bsf, bt)
    corr, _ = M.pressure_rhs(sf, cc, w, gamma, g, phi, bcell, bphi)
    M.pressure_flux(up, corr, b, phi, cc, bcell, bsf, bcf, bg, bt, bphi)
    M.fv_div(phi, bcell, bphi)
    M.prepare(dg, up, 2)
    xi = M.to_internal(b)
    M.amul_prepared(xi)
    M.amul_prepared(xi.float())
    # GAMG with the two-stage Gauss-Seidel smoother on algebraic pairing weights
    from paper_2512_22215_gb300 import GamgSolver
    gs = GamgSolver(M, up.abs(), smoother=1)
    _, pg = gs.solve(dg, up, b, None, SolverControls(tolerance=1e-8, max_iter=500))
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": f"{args.n}^3", "cells": m.n_cells, "faces": m.n_faces,
                      "mixed_iters": pm["n_iter"], "fp64_iters": pf["n_iter"], "gamg_vcycles": pg["n_iter"]}),
          flush=True)


def cpu_sample(case, n_inner_sample: int):
    """The oracle as it stands on the host cores: assembly, DIC factor, one FP64
    residual and `n_inner_sample` FP32 inner iterations of the refinement,
    projected to the workload's iteration counts.  Returns (ms per step, info)."""
    import numpy as np
    import oracle
    m = case.mesh
    t0 = time.perf_counter()
    up, dg = oracle.assemble_laplacian(m, case.gamma, case.bgamma, case.btype)
    t_asm = time.perf_counter() - t0
    # mixed_ir with one outer step runs: factor, 2 FP64 residuals and k inner iterations
    t0 = time.perf_counter()
    oracle.mixed_ir(m.lower, m.upper_addr, dg, up, case.b, tol=1e-8, max_iter=2, max_outer=1)
    t_a = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.mixed_ir(m.lower, m.upper_addr, dg, up, case.b, tol=1e-8, max_iter=2 + n_inner_sample, max_outer=1)
    t_b = time.perf_counter() - t0
    per_inner = (t_b - t_a) / n_inner_sample
    fixed = t_a - 2 * per_inner                           # factor + 2 residuals + setup
    t0 = time.perf_counter()
    oracle.amul(m.lower, m.upper_addr, dg, up, case.b)
    t_res = time.perf_counter() - t0
    proj = t_asm + fixed + max(0, PROJECTION_ITERS["outer"] - 1) * t_res + PROJECTION_ITERS["inner"] * per_inner
    sample = (f"oracle (restarted mixed form, one refinement step): assembly + DIC factor + 2 FP64 residuals + "
              f"{2 + n_inner_sample} FP32 iterations (two timed runs, per-iteration cost by difference), "
              f"projected to {PROJECTION_ITERS['inner']} FP32 iterations and {PROJECTION_ITERS['outer']} FP64 "
              f"residuals (the GPU's counts for this workload)")
    return proj * 1e3, dict(sample=sample, per_inner_ms=per_inner * 1e3, assembly_ms=t_asm * 1e3,
                            cpu_seconds=t_asm + t_a + t_b + t_res)


def run_reference(args, rank, world):
    """The oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    case = make_case(args.n, args.seed)
    cores = 1
    vals = []
    info = {}
    for k in range(args.warmup + args.steps):
        v, info = cpu_sample(case, max(2, args.cpu_iters // 2))
        if k >= args.warmup:
            vals.append(v)
    vals.sort()
    value = vals[len(vals) // 2]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed)", "data": "synthetic",
        "config": config_of(case, args),
        "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle, projected",
                         "sample": info["sample"]},
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(case, args):
    m = case.mesh
    return {"workload": f"{args.n}^3 jittered permuted hex mesh, log-normal gamma, DIC, tol 1e-8",
            "cells": m.n_cells, "faces": m.n_faces, "precond": "DIC", "tolerance": 1e-8,
            "l2": "inputs larger than L2 (workspace and per-iteration streams > 129 MB)"}


def batch_measure(dev, steps: int):
    """64 independent systems (jittered, permuted hex blocks, side lengths from
    cell counts log-uniform in 1e4..5e5, seed 5) in one persistent launch
    replayed from a CUDA graph, FP64 and mixed, autotuned block size, split
    weights and grid.  Returns the figures for the JSON line."""
    import numpy as np
    import torch
    import hexmesh
    from paper_2512_22215_gb300 import MIXED, BatchSolve, LduMesh, SolverControls
    sides = hexmesh.batch_sizes(64, seed=5)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Ms, D, U, B, X = [], [], [], [], []
    for k, n in enumerate(sides):
        c = hexmesh.pressure_case(n, jitter=0.2, permute=True, seed=500 + k, lognormal_gamma=True)
        m = c.mesh
        M = LduMesh(m.lower, m.upper_addr, m.n_cells, device=dev, centres=m.c)
        up, dg = M.assemble_laplacian(T(m.sf), T(m.c), T(c.gamma), T(m.bface_cell), T(m.bface_sf), T(m.bface_cf),
                                      T(c.bgamma), T(c.btype))
        Ms.append(M)
        D.append(dg)
        U.append(up)
        B.append(T(c.b))
        X.append(torch.zeros(m.n_cells, dtype=torch.float64, device=dev))
    cells = sum(M.n_cells for M in Ms)
    out = {"n_sys": len(Ms), "cells": cells}
    for name, ctl in [("fp64", SolverControls(precond=2, tolerance=1e-8)),
                      ("mixed", SolverControls(precond=2, precision=MIXED, tolerance=1e-8))]:
        bs = BatchSolve(Ms, D, U, B, X, ctl, autotune=True)
        for x in X:
            x.zero_()
        bs.run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(3, steps)):
            for x in X:
                x.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            bs.run()
            c.record()
            c.synchronize()
            ts.append(a.elapsed_time(c))
        res = bs.results()
        ts.sort()
        out[name] = {"ms": round(ts[len(ts) // 2], 3), "max_iters": max(r["n_iter"] for r in res),
                     "all_converged": all(r["converged"] == 1 for r in res),
                     "max_true_rel_residual_l2": max(r["true_rel_residual_l2"] for r in res),
                     "block_threads": bs.block_threads, "grid_blocks": bs.grid_blocks,
                     "graph_captured": bs.graph_captured, "tuned_ms": round(bs.tuned_ms, 3),
                     "tuner_trials": bs.trials}
        del bs
    return out


def run_batch(args, rank, world, local):
    """The batched workload alone, as a line of its own."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    out = batch_measure(torch.device("cuda", local), args.steps)
    line = {"metric": "batched PCG time to 1e-8, 64 systems", "value": out["mixed"]["ms"], "unit": "ms",
            "higher_is_better": False, "n_gpus": world, "steps": args.steps, "data": "synthetic",
            "config": {"workload": "64 jittered permuted hex blocks, cells log-uniform in 1e4..5e5, seed 5",
                       "cells": out["cells"]}, "fp64": out["fp64"], "mixed": out["mixed"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def measured_oracle_solve(dev):
    """A full oracle solve timed to the end (no projection) beside the GPU's on
    the same system: 64^3 jittered, permuted, log-normal gamma, seed 4, FP64
    DIC-PCG to 1e-8, one host core."""
    import numpy as np
    import torch
    import hexmesh
    import oracle
    from paper_2512_22215_gb300 import LduMesh, SolverControls
    c = hexmesh.pressure_case(64, jitter=0.2, permute=True, seed=4, lognormal_gamma=True)
    m = c.mesh
    up, dg = oracle.assemble_laplacian(m, c.gamma, c.bgamma, c.btype)
    t0 = time.perf_counter()
    _, po = oracle.pcg(m.lower, m.upper_addr, dg, up, c.b, precond=2, tol=1e-8)
    t_cpu = time.perf_counter() - t0
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M = LduMesh(m.lower, m.upper_addr, m.n_cells, device=dev, centres=m.c)
    d, u, b = T(dg), T(up), T(c.b)
    x = torch.zeros_like(b)
    ctl = SolverControls(precond=2, tolerance=1e-8)
    M.solve(d, u, b, x, ctl)
    ts = []
    for _ in range(5):
        x.zero_()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, pg = M.solve(d, u, b, x, ctl)
        e.record()
        e.synchronize()
        ts.append(a.elapsed_time(e))
    ts.sort()
    return {"workload": "64^3 jittered permuted hex mesh, log-normal gamma, seed 4, FP64 DIC-PCG to 1e-8",
            "oracle_ms": round(t_cpu * 1e3, 1), "oracle_iters": po["n_iter"], "cores": 1,
            "gpu_ms": round(ts[2], 3), "gpu_iters": pg["n_iter"], "ratio": round(t_cpu * 1e3 / ts[2], 1)}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.batch:
        run_batch(args, rank, world, local)
        return
    if args.profile_run:
        if rank == 0:
            profile_run(args, local)
        return
    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    host_affinity = bind_to_gpu_cpus(local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_22215_gb300 import MIXED, LduMesh, SolverControls, lib
    from paper_2512_22215_gb300.core import perf_tensor, read_perf

    case = make_case(args.n, args.seed)
    m = case.mesh
    N, F = m.n_cells, m.n_faces
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M = LduMesh(m.lower, m.upper_addr, N, device=dev, centres=m.c, asymmetric=True)
    sf, cc, bcell, bsf, bcf, bg, bt = T(m.sf), T(m.c), T(m.bface_cell), T(m.bface_sf), T(m.bface_cf), \
        T(case.bgamma), T(case.btype)
    gamma, b = T(case.gamma), T(case.b)
    x = torch.zeros(N, dtype=torch.float64, device=dev)
    perf = perf_tensor(1, dev)
    ctl_mixed = SolverControls(precond=2, precision=MIXED, tolerance=1e-8, inner_rel_tol=1e-2)
    ctl_f64 = SolverControls(precond=2, tolerance=1e-8)
    s = torch.cuda.current_stream()

    def step(ctl):
        up, dg = M.assemble_laplacian(sf, cc, gamma, bcell, bsf, bcf, bg, bt)
        x.zero_()
        M.solve(dg, up, b, x, ctl, perf=perf)
        return up, dg

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- warm-up
    for _ in range(max(3, args.warmup)):
        up, dg = step(ctl_mixed)
    barrier()
    p_mixed = read_perf(perf)[0]

    # ------------------------------------------------------------ timed region
    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    n0 = lib().spuma_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        step(ctl_mixed)
    e1.record(s)
    barrier()
    launches = lib().spuma_launch_count() - n0
    ms_step = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    ms_step_max = reduce_max(ms_step, world, dev)

    # ----------------------------------------------------- end to end (host)
    gamma_h = torch.from_numpy(case.gamma).pin_memory()
    b_h = torch.from_numpy(case.b).pin_memory()
    x_h = torch.empty(N, dtype=torch.float64).pin_memory()
    perf_h = torch.empty(perf.numel(), dtype=torch.uint8).pin_memory()
    gamma_d, b_d = torch.empty_like(gamma), torch.empty_like(b)

    def e2e_step(marks=None):
        """One end-to-end step; `marks` (4 events) split it into host-to-device
        copies, assembly, solve and device-to-host copies."""
        gamma_d.copy_(gamma_h, non_blocking=True)
        b_d.copy_(b_h, non_blocking=True)
        if marks:
            marks[0].record(s)
        u2, d2 = M.assemble_laplacian(sf, cc, gamma_d, bcell, bsf, bcf, bg, bt)
        if marks:
            marks[1].record(s)
        x.zero_()
        M.solve(d2, u2, b_d, x, ctl_mixed, perf=perf)
        if marks:
            marks[2].record(s)
        x_h.copy_(x, non_blocking=True)
        perf_h.copy_(perf, non_blocking=True)
        if marks:
            marks[3].record(s)

    e2e_step()
    # sampled like the timed steps (the same settle time after the sampler starts)
    clocks_e2e = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    a.record(s)
    for k in range(args.steps):
        e2e_step(marks[k])
    c.record(s)
    c.synchronize()
    clk_e2e = clocks_e2e.stop()
    e2e_ms = reduce_max(a.elapsed_time(c) / args.steps, world, dev)
    # per-stage split of the end-to-end steps (CUDA events on the same stream)
    starts = [a] + [mk[3] for mk in marks[:-1]]
    split = {"h2d_ms": [], "assembly_ms": [], "solve_ms": [], "d2h_ms": []}
    for st, mk in zip(starts, marks):
        split["h2d_ms"].append(st.elapsed_time(mk[0]))
        split["assembly_ms"].append(mk[0].elapsed_time(mk[1]))
        split["solve_ms"].append(mk[1].elapsed_time(mk[2]))
        split["d2h_ms"].append(mk[2].elapsed_time(mk[3]))
    e2e_split = {k: round(sum(v) / len(v), 3) for k, v in split.items()}
    e2e_split["max_step_ms"] = round(max(st.elapsed_time(mk[3]) for st, mk in zip(starts, marks)), 3)
    h2d = gamma_h.numel() * 8 + b_h.numel() * 8
    d2h = x_h.numel() * 8 + perf_h.numel()

    # solve kernel alone (mixed and FP64), CUDA events around the launch
    def time_solve(ctl, reps):
        ts = []
        for _ in range(reps):
            x.zero_()
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            M.solve(dg, up, b, x, ctl, perf=perf)
            c.record(s)
            c.synchronize()
            ts.append(a.elapsed_time(c))
        ts.sort()
        return ts[len(ts) // 2], read_perf(perf)[0]

    up, dg = M.assemble_laplacian(sf, cc, gamma, bcell, bsf, bcf, bg, bt)
    solve_mixed_ms, p_mixed = time_solve(ctl_mixed, max(3, args.steps))
    solve_f64_ms, p_f64 = time_solve(ctl_f64, max(3, args.steps))
    # assembly + FP64 solve per step (the comparison arm of the metric)
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(args.steps):
        step(ctl_f64)
    c.record(s)
    c.synchronize()
    f64_step_ms = a.elapsed_time(c) / args.steps

    # stand-alone Amul on the prepared matrix (the PCG's Amul phase)
    M.prepare(dg, up, 2)
    xi = M.to_internal(b)
    yi = torch.empty_like(xi)
    xi32, yi32 = xi.float(), torch.empty(N, dtype=torch.float32, device=dev)

    def time_amul(xv, yv, reps=50):
        """Back-to-back launches between two events: the GPU never waits for
        the host between them, so the average is the kernel's own time."""
        for _ in range(3):
            M.amul_prepared(xv, yv)
        torch.cuda.synchronize()
        a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(s)
        for _ in range(reps):
            M.amul_prepared(xv, yv)
        c_.record(s)
        c_.synchronize()
        return a_.elapsed_time(c_) / reps * 1e3   # us

    amul64_us = time_amul(xi, yi)
    amul32_us = time_amul(xi32, yi32)

    # the pressure-correction step's explicit operators around the solve
    # (gradient, corrected-laplacian RHS, flux reconstruction, divergence)
    def time_op(fn, reps=20):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(s)
        for _ in range(reps):
            fn()
        c_.record(s)
        c_.synchronize()
        return a_.elapsed_time(c_) / reps * 1e3   # us

    rng_ps = np.random.default_rng(7)
    cf_d, v_d = T(m.cf), T(m.v)
    phi_d = T(rng_ps.standard_normal(F) * np.linalg.norm(m.sf, axis=1))
    bphi_d = T(rng_ps.standard_normal(m.n_bfaces) * np.linalg.norm(m.bface_sf, axis=1))
    w_d = M.fv_weights(sf, cf_d, cc)
    g_d = M.fv_grad(sf, w_d, v_d, b, bcell, bsf, bt)
    corr_d, rhs_d = M.pressure_rhs(sf, cc, w_d, gamma, g_d, phi_d, bcell, bphi_d)
    B = m.n_bfaces
    ps_us = {"grad": time_op(lambda: M.fv_grad(sf, w_d, v_d, b, bcell, bsf, bt)),
             "rhs": time_op(lambda: M.pressure_rhs(sf, cc, w_d, gamma, g_d, phi_d, bcell, bphi_d)),
             "flux": time_op(lambda: M.pressure_flux(up, corr_d, b, phi_d, cc, bcell, bsf, bcf, bg, bt, bphi_d)),
             "div": time_op(lambda: M.fv_div(phi_d, bcell, bphi_d))}
    ps_bytes = {"grad": 40 * F + 40 * N + 29 * B, "rhs": 72 * F + 56 * N + 12 * B,
                "flux": 40 * F + 8 * N + 77 * B, "div": 8 * F + 8 * N + 12 * B}

    # PBiCG with DILU on an asymmetric system of the same mesh: the laplacian
    # plus first-order upwind convection of a seeded face flux (Peclet 2),
    # diagonal = row |off-diagonal| sum (+ Dirichlet) / 0.7 (the paper's U
    # under-relaxation), tolerance 1e-8, FP64
    a_d = -up
    phi_c = 2.0 * torch.from_numpy(rng_ps.standard_normal(F)).to(dev) * a_d.mean()
    lower_c = -a_d - torch.clamp(phi_c, min=0.0)
    upper_c = -a_d - torch.clamp(-phi_c, min=0.0)
    lo_i, up_i = M.lower.long(), M.upper_addr.long()
    rowabs = torch.zeros(N, dtype=torch.float64, device=dev)
    rowabs.index_add_(0, up_i, lower_c.abs())
    rowabs.index_add_(0, lo_i, upper_c.abs())
    lap = torch.zeros(N, dtype=torch.float64, device=dev)
    lap.index_add_(0, lo_i, a_d)
    lap.index_add_(0, up_i, a_d)
    diag_c = (rowabs + (dg - lap)) / 0.7
    ctl_bicg = SolverControls(precond=3, tolerance=1e-8)
    xb = torch.zeros(N, dtype=torch.float64, device=dev)
    M.pbicg_solve(diag_c, lower_c, upper_c, b, xb, ctl_bicg, perf=perf)
    torch.cuda.synchronize()
    bicg_ts = []
    for _ in range(3):
        xb.zero_()
        a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(s)
        M.pbicg_solve(diag_c, lower_c, upper_c, b, xb, ctl_bicg, perf=perf)
        c_.record(s)
        c_.synchronize()
        bicg_ts.append(a_.elapsed_time(c_))
    bicg_ms = sorted(bicg_ts)[1]
    p_bicg = read_perf(perf)[0]
    bicg_bytes = p_bicg["n_iter"] * (280 * N + 96 * F)
    # the same system with a fixed 100 iterations (tolerance 0), so that the
    # iterations, not the setup (gather, DILU factor), dominate the time
    ctl_fixed = SolverControls(precond=3, tolerance=0.0, max_iter=100, min_iter=100)
    fixed_ts = []
    for _ in range(3):
        xb.zero_()
        a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(s)
        M.pbicg_solve(diag_c, lower_c, upper_c, b, xb, ctl_fixed, perf=perf)
        c_.record(s)
        c_.synchronize()
        fixed_ts.append(a_.elapsed_time(c_))
    fixed_ms = sorted(fixed_ts)[1]
    p_fixed = read_perf(perf)[0]

    # GAMG (the paper's production pressure solver) on the bench system, FP64
    # to 1e-8: hierarchy built once from |S_f| (host), then timed solves
    from paper_2512_22215_gb300 import GamgSolver
    t_h = time.time()
    gs = GamgSolver(M, torch.linalg.norm(sf, dim=1))
    gamg_setup_s = time.time() - t_h
    ctl_gamg = SolverControls(tolerance=1e-8, max_iter=500)
    xg = torch.zeros(N, dtype=torch.float64, device=dev)
    gs.solve(dg, up, b, xg, ctl_gamg, perf=perf)
    torch.cuda.synchronize()
    gamg_ts = []
    for _ in range(3):
        xg.zero_()
        a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(s)
        gs.solve(dg, up, b, xg, ctl_gamg, perf=perf)
        c_.record(s)
        c_.synchronize()
        gamg_ts.append(a_.elapsed_time(c_))
    gamg_ms = sorted(gamg_ts)[1]
    p_gamg = read_perf(perf)[0]
    del gs
    # the same with algebraic pairing weights |upper_f| (the caller's choice of face weight)
    gs2 = GamgSolver(M, up.abs())
    xg.zero_()
    gs2.solve(dg, up, b, xg, ctl_gamg, perf=perf)
    torch.cuda.synchronize()
    xg.zero_()
    a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_.record(s)
    gs2.solve(dg, up, b, xg, ctl_gamg, perf=perf)
    c_.record(s)
    c_.synchronize()
    gamg2_ms = a_.elapsed_time(c_)
    p_gamg2 = read_perf(perf)[0]
    # the paper's smoother table on the same hierarchy: Richardson or two-stage
    # Gauss-Seidel, diagonal or DIC preconditioning of the coarsest level's PCG
    gamg_options = {}
    for smoother, sname in ((0, "richardson"), (1, "gauss_seidel_2stage")):
        for coarsest, cname in ((1, "diagonal"), (2, "dic")):
            gs2.set_options(smoother, coarsest)
            xg.zero_()
            gs2.solve(dg, up, b, xg, ctl_gamg, perf=perf)
            torch.cuda.synchronize()
            xg.zero_()
            a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(s)
            gs2.solve(dg, up, b, xg, ctl_gamg, perf=perf)
            c_.record(s)
            c_.synchronize()
            po = read_perf(perf)[0]
            gamg_options[f"{sname}+{cname}"] = {"solve_ms": round(a_.elapsed_time(c_), 3), "iters": po["n_iter"],
                                                "converged": po["converged"],
                                                "true_rel_residual_l2": po["true_rel_residual_l2"]}
    del gs2

    # the batched form: 64 systems, ~8.2M cells in total, one persistent launch per solve
    batch_out = batch_measure(dev, args.steps)

    # -------------------------------------------------------------- roofline
    wb = workload_bytes(N, F)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    mixed_bytes = p_mixed["n_iter"] * wb["it32"] + (p_mixed["n_outer"] + 1) * wb["resid64"]
    achieved = mixed_bytes / (solve_mixed_ms * 1e-3) / 1e9
    f64_bytes = p_f64["n_iter"] * wb["it64"]
    roofline = {"kernel": "k_solve (persistent mixed-precision solve, one launch per solve)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "peak_kind": peak_kind,
                "traffic": traffic_bytes(N, F, p_mixed["n_iter"], p_mixed["n_outer"]),
                "algorithmic_bytes": int(mixed_bytes),
                "basis": "inner iterations x (76N + 36F) + (outer + 1) FP64 residuals x (16F + 40N)"}

    line = {
        "metric": METRIC, "value": round(ms_step_max, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step_max, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed)", "data": "synthetic",
        "config": config_of(case, args),
        "step": "laplacian assembly + mixed-precision DIC-PCG solve to 1e-8",
        "mixed": {"solve_ms": round(solve_mixed_ms, 3), "inner_iters": p_mixed["n_iter"],
                  "outer": p_mixed["n_outer"], "final_residual": p_mixed["final_residual"],
                  "converged": p_mixed["converged"]},
        "fp64": {"solve_ms": round(solve_f64_ms, 3), "step_ms": round(f64_step_ms, 3), "iters": p_f64["n_iter"],
                 "final_residual": p_f64["final_residual"], "converged": p_f64["converged"],
                 "achieved_gbs": round(f64_bytes / (solve_f64_ms * 1e-3) / 1e9, 1)},
        "mixed_speedup_vs_fp64": round(solve_f64_ms / solve_mixed_ms, 3),
        "amul": {"f64_us": round(amul64_us, 2), "f64_gbs_ldu": round(wb["amul64"] / amul64_us / 1e3, 1),
                 "f64_frac_ldu": round(wb["amul64"] / amul64_us / 1e3 / hbm, 4),
                 "f32_us": round(amul32_us, 2), "f32_gbs_ldu": round(wb["amul32"] / amul32_us / 1e3, 1),
                 "basis": "LDU algorithmic bytes 16F + 24N (FP64), 12F + 12N (FP32)"},
        "pressure_step": dict(
            **{f"{k}_us": round(v, 2) for k, v in ps_us.items()},
            **{f"{k}_gbs": round(ps_bytes[k] / ps_us[k] / 1e3, 1) for k in ps_us},
            basis="algorithmic bytes, int32 indices: grad 40F + 40N + 29B, rhs 72F + 56N + 12B, "
                  "flux 40F + 8N + 77B, div 8F + 8N + 12B (B boundary faces); the per-cell "
                  "boundary-face lists are built on the first call and reused"),
        "pbicg": {"solve_ms": round(bicg_ms, 3), "iters": p_bicg["n_iter"],
                  "final_residual": p_bicg["final_residual"], "converged": p_bicg["converged"],
                  "status": p_bicg["status"], "achieved_gbs": round(bicg_bytes / (bicg_ms * 1e-3) / 1e9, 1),
                  "basis": "per iteration 280N + 96F bytes (two DILU applications, Amul + Tmul, two "
                           "search directions, x/rA/rT update, FP64)",
                  "system": "laplacian + upwind convection (Peclet 2), diagonal / 0.7, DILU, tol 1e-8",
                  "fixed_100_iterations": {
                      "solve_ms": round(fixed_ms, 3), "iters": p_fixed["n_iter"],
                      "per_iteration_us": round((fixed_ms - bicg_ms) / max(1, p_fixed["n_iter"] - p_bicg["n_iter"])
                                                * 1e3, 1),
                      "achieved_gbs": round((280 * N + 96 * F) / ((fixed_ms - bicg_ms) * 1e-3 /
                                            max(1, p_fixed["n_iter"] - p_bicg["n_iter"])) / 1e9, 1),
                      "basis": "(solve_ms - tolerance solve's ms) / (100 - its iterations): the setup cancels"}},
        "gamg": {"solve_ms": round(gamg_ms, 3), "iters": p_gamg["n_iter"],
                 "final_residual": p_gamg["final_residual"], "converged": p_gamg["converged"],
                 "status": p_gamg["status"], "levels": p_gamg["n_levels"],
                 "hierarchy_setup_s": round(gamg_setup_s, 2),
                 "system": "the bench system (laplacian, DIC-PCG's), FP64 GAMG to 1e-8, Richardson smoothing, "
                           "pairing weights |S_f| (face area, OpenFOAM's default agglomeration)",
                 "algebraic_weights": {"solve_ms": round(gamg2_ms, 3), "iters": p_gamg2["n_iter"],
                                       "converged": p_gamg2["converged"],
                                       "weights": "|upper_f| (algebraic pairing)",
                                       "smoother_x_coarsest": gamg_options}},
        "n_levels": M.n_levels,
        "batch": batch_out,
        "roofline": roofline,
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "spuma_assemble_laplacian + spuma_pcg_solve with gamma and b copied from pinned host "
                       "memory and x and the solver report copied back, every step",
                "clocks": clk_e2e, "host_affinity": host_affinity, "split": e2e_split},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu:
        cpu_ms, info = cpu_sample(case, args.cpu_iters)
        line["cpu_baseline"] = {"value": round(cpu_ms, 1), "unit": "ms", "cores": 1, "kind": "oracle, projected",
                                "sample": info["sample"], "per_inner_iteration_ms": round(info["per_inner_ms"], 1),
                                "cpu_seconds": round(info["cpu_seconds"], 1),
                                "coe": round(cpu_ms / ms_step_max, 1),
                                "measured_full_solve": measured_oracle_solve(dev)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
