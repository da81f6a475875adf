#!/usr/bin/env python
"""HPG-MxP benchmark on GB300: mixed-precision GMRES-IR GFLOP/s and time to a
1e-9 relative residual, against the same library's FP64-only solve.

One step = one full GMRES-IR solve from x0 = 0 to ||b - A x|| / ||b|| < 1e-9
on the 128^3 workload (b = A*1 + N(0, 1e-3^2) noise, seed 0, nonsymmetric
stencil beta = 0.5, GMRES(30), 4-level V-cycle with 1+1 symmetric
Gauss-Seidel sweeps).  Inputs are resident in HBM when the timed region
starts; the e2e figure repeats the solve through the C ABI with pinned host
buffers, the copies inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
replica (the path has no data-parallel exchange on one problem), timing is
the max over ranks and `value` sums the ranks' flops.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GMRES-IR GFLOP/s and time-to-1e-9 residual, MxP vs FP64, 1 GB300; % HBM peak"
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per launch of the level-0 FP32 Gauss-Seidel phase
# kernel at 128^3, from one ncu capture of that kernel, valid while the
# kernel's source text (the kernel and the helpers it inlines) hashes to
# `sources_sha256`.
GS_TRAFFIC = {"workload": "mxp_gmres30_128cube", "bytes_per_launch": 65166976.0,
              "sources_sha256": "d797e9973fb181b4d5383dbc69dd6b586e4b41f70cf2ba667a9760cb975d6a1a"}
# (file, first line of the block, text that ends it): the kernel's source
GS_KERNEL_TEXT = (
    ("paper_2507_11512_gb300/csrc/sparse.cu", "template <typename T> struct PhaseRows;",
     "// One Gauss-Seidel colour phase"),
    ("paper_2507_11512_gb300/csrc/sparse.cu", "template <typename T, bool STREAM, int MC>",
     "// The bandwidth-variant instantiation"),
    ("paper_2507_11512_gb300/csrc/hpg_internal.cuh", "template <bool STREAM, typename V>", "\n}\n"),
    ("paper_2507_11512_gb300/csrc/hpg_internal.cuh",
     "__host__ __device__ constexpr unsigned gs_slot_mask", "\n}\n"),
    ("paper_2507_11512_gb300/csrc/hpg_internal.cuh",
     "template <typename V>\n__device__ __forceinline__ V ld_dep", "\n}\n"),
)


def gs_sources_sha256():
    """sha256 of the Gauss-Seidel phase kernel's source blocks (None if a
    block is not found)."""
    import hashlib
    h = hashlib.sha256()
    for rel, start, end in GS_KERNEL_TEXT:
        with open(os.path.join(ROOT, rel)) as f:
            text = f.read()
        i = text.find(start)
        j = text.find(end, i + len(start)) if i >= 0 else -1
        if i < 0 or j < 0:
            return None
        h.update(text[i:j + len(end)].encode())
    return h.hexdigest()


def gs_traffic(workload="mxp_gmres30_128cube"):
    """Captured DRAM traffic per launch, or None if the kernel changed since
    (or the capture was of another workload)."""
    if GS_TRAFFIC["bytes_per_launch"] is None or workload != GS_TRAFFIC["workload"]:
        return None
    sha = gs_sources_sha256()
    return GS_TRAFFIC["bytes_per_launch"] if sha and sha == GS_TRAFFIC["sources_sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="mxp_gmres30_128cube")
    ap.add_argument("--basis", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="storage of the Krylov basis in the mixed-precision solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--validation", default="standard", choices=["standard", "fullscale"],
                    help="validation phase for the penalty n_d/n_ir (Sec. 3, Sec. 3.3)")
    ap.add_argument("--nd-max", type=int, default=10000,
                    help="FP64 iteration cap of the validation phase")
    ap.add_argument("--cpu-sample-iters", type=int, default=8)
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def reduce_max_sum(values, op_list, backend_device=None):
    """All-reduce a list of floats with per-entry MAX or SUM (single process:
    identity).  Used for the max-over-ranks time and summed flops."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    out = []
    for v, op in zip(values, op_list):
        t = torch.tensor([float(v)], dtype=torch.float64, device=backend_device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
        out.append(float(t.item()))
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", FALLBACK_HBM_GBS), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_sample(workload_name, iters, threads=1):
    """Times the FP64 CPU oracle on a bounded sample of the workload in a
    child process: `iters` inner GMRES steps (or the whole solve, if it takes
    fewer), with `threads` BLAS threads (None: the library's default, all
    cores)."""
    code = r"""
import json, os, sys, time
sys.path.insert(0, %r)
import numpy as np
from oracle import hpg_oracle as O
from workloads import WORKLOADS, x_true, rhs_noise
w = WORKLOADS[%r]
t0 = time.perf_counter()
lv = O.build_hierarchy(*w.dims, levels=w.levels, beta=w.beta)
n = lv[0].n
b = lv[0].A @ x_true(n) + rhs_noise(n, w.noise_std, w.seed)
t1 = time.perf_counter()
x, info = O.gmres_ir(lv, b, tol=w.tol, restart=w.restart, maxit=%d)
t2 = time.perf_counter()
cyc = []
left = info.iterations
while left > 0:
    cyc.append(min(left, w.restart)); left -= cyc[-1]
fl = O.solve_flops(lv, cyc)
print(json.dumps({"seconds": t2 - t1, "setup_s": t1 - t0, "flops": fl,
                  "iterations": info.iterations}))
""" % (ROOT, workload_name, iters)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if threads is None:
            env.pop(k, None)
        else:
            env[k] = str(threads)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed: " + p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------- reference arm
def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from workloads import WORKLOADS
    w = WORKLOADS[args.workload]
    iters = max(1, args.cpu_sample_iters // 4)
    times, flops = [], []
    for step in range(args.warmup + args.steps):
        r = oracle_sample(args.workload, iters)
        if step >= args.warmup:
            times.append(r["seconds"])
            flops.append(r["flops"])
    gfl = sum(flops) / sum(times) / 1e9
    sample = ("%d inner GMRES steps of the %s workload per step (FP64 oracle, numpy/scipy, "
              "hierarchy build untimed)" % (iters, w.name))
    line = {"impl": "reference", "metric": METRIC, "value": gfl, "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.dims), "beta": w.beta,
                       "restart": w.restart, "tol": w.tol},
            "cpu_baseline": {"value": gfl, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gfl, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rounded(v, digits=5):
    """Floats rounded to `digits` significant digits (a shorter JSON line)."""
    if isinstance(v, float):
        return float("%.*g" % (digits, v))
    if isinstance(v, dict):
        return {k: rounded(x, digits) for k, x in v.items()}
    if isinstance(v, list):
        return [rounded(x, digits) for x in v]
    return v


# ------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_11512_gb300 as hpg
    from paper_2507_11512_gb300 import metrics
    from workloads import WORKLOADS, rhs_noise

    w = WORKLOADS[args.workload]
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    prob = hpg.Problem(*w.dims, beta=w.beta, levels=w.levels, pre_sweeps=w.pre,
                       post_sweeps=w.post)
    dims_list = metrics.level_dims(w.dims, w.levels)
    n = w.n
    # b = A * 1 + e (FP64), formed with the library's FP64 SpMV
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    ax = prob.to_natural(prob.spmv(prob.to_storage(ones)))
    b = ax + torch.tensor(rhs_noise(n, w.noise_std, w.seed), device=dev)
    x = torch.zeros_like(b)

    basis_mxp = {"fp32": hpg.HPG_FP32, "bf16": hpg.HPG_BF16, "fp16": hpg.HPG_FP16}[args.basis]

    def solve(inner):
        x.zero_()
        return hpg.gmres_ir_solve(prob.h, b, x, tol=w.tol, restart=w.restart, maxit=w.maxit,
                                  inner=inner,
                                  basis=basis_mxp if inner == hpg.HPG_FP32 else inner)

    def timed(inner, steps, warmup):
        for _ in range(warmup):
            solve(inner)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for _ in range(steps):
            infos.append(solve(inner))
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        return ms, infos

    sampler = ClockSampler(local_rank)
    # ---- mixed precision (headline)
    for _ in range(args.warmup):
        solve(hpg.HPG_FP32)
    sampler.start()
    ms, infos = timed(hpg.HPG_FP32, args.steps, 0)
    clocks = sampler.stop()
    for inf in infos:
        assert inf["status"] == 0 and inf["rel_residual"] < w.tol, inf
    flops = sum(metrics.solve_flops(dims_list, metrics.cycles_from_info(
        i["iterations"], i["restarts"], w.restart)) for i in infos)
    launches = sum(i["kernel_launches"] for i in infos)
    ms_max, flops_sum = reduce_max_sum([ms, flops], ["max", "sum"], dev)
    gflops = flops_sum / (ms_max / 1e3) / 1e9
    n_ir = infos[-1]["iterations"]

    x_mxp = x.clone()   # the mixed-precision solution of the last timed solve

    # ---- FP64-only solve of the same code (Algorithm 2 as the paper's "double")
    fp64 = None
    if not args.no_fp64:
        ms64, infos64 = timed(hpg.HPG_FP64, max(1, args.steps // 2), 1)
        err_vs_fp64 = (torch.linalg.norm(x_mxp - x) / torch.linalg.norm(x)).item()
        fl64 = sum(metrics.solve_flops(dims_list, metrics.cycles_from_info(
            i["iterations"], i["restarts"], w.restart)) for i in infos64)
        ms64_max, fl64_sum = reduce_max_sum([ms64, fl64], ["max", "sum"], dev)
        n_d = infos64[-1]["iterations"]
        fp64 = {"value": fl64_sum / (ms64_max / 1e3) / 1e9, "unit": "GFLOP/s",
                "ms_per_solve": ms64_max / len(infos64), "iterations": n_d,
                "rel_residual": infos64[-1]["rel_residual"],
                "mxp_solution_rel_diff": err_vs_fp64}

    # ---- validation phase: n_d (FP64 GMRES) and n_ir (GMRES-IR) for the penalty
    valid = None
    if not args.no_fp64:
        from paper_2507_11512_gb300 import validation

        def vsolve(prec, tol, maxit):
            x.zero_()
            inner = hpg.HPG_FP64 if prec == "fp64" else hpg.HPG_FP32
            return hpg.gmres_ir_solve(prob.h, b, x, tol=tol, restart=w.restart, maxit=maxit,
                                      inner=inner,
                                      basis=basis_mxp if inner == hpg.HPG_FP32 else inner)
        valid = validation.validate(vsolve, args.validation, w.tol, args.nd_max)

    # ---- per-kernel profile of one MxP solve (CUDA events on the solve's stream)
    hpg.set_profiling(prob.h, True)
    solve(hpg.HPG_FP32)
    torch.cuda.synchronize()
    prof = hpg.profile_report(prob.h)
    hpg.set_profiling(prob.h, False)
    tot_ms = sum(p["total_ms"] for p in prof)
    prof.sort(key=lambda p: -p["total_ms"])
    peak, peak_src = measured_peaks()

    # ---- dominant kernel (level-0 FP32 Gauss-Seidel phase) timed with CUDA
    # events on the launching stream, launched exactly as the V-cycle launches
    # it: hpg_mg_smooth = 15 colour phases per sweep (colours 0..7, 6..0).
    # Between sweeps the level-0 FP32 SpMV streams the whole matrix (453 MB,
    # evict-first) as it does after every V-cycle of the solve, so that no
    # phase finds the slice the previous sweep left in L2; only the sweeps
    # are timed.
    gs_reps = 20
    info0 = prob.info[0]
    r_gs = prob.to_storage(torch.randn(n, dtype=torch.float64, device=dev,
                                       generator=torch.Generator(device=dev).manual_seed(1)),
                           dtype=torch.float32)
    z_gs = torch.zeros_like(r_gs)
    w_gs = torch.empty_like(r_gs)
    for _ in range(3):
        hpg.spmv(prob.h, 0, r_gs, w_gs)
        hpg.mg_smooth(prob.h, 0, r_gs, z_gs, 1, False)
    torch.cuda.synchronize()
    # both captured in CUDA graphs, as the solve launches them
    g_spmv, g_sweep = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_spmv):
        hpg.spmv(prob.h, 0, r_gs, w_gs)
    with torch.cuda.graph(g_sweep):
        hpg.mg_smooth(prob.h, 0, r_gs, z_gs, 1, False)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(gs_reps)]
    for a, c in ev:
        g_spmv.replay()
        a.record(stream)
        g_sweep.replay()
        c.record(stream)
    torch.cuda.synchronize()
    gs_ms = sum(a.elapsed_time(c) for a, c in ev)
    del g_spmv, g_sweep
    cnt = info0["colour_count"]
    gs_row_bytes = metrics.gs_row_bytes(4, 4)
    gs_phases = 15
    gs_bytes = (sum(cnt) + sum(cnt[:7])) * gs_row_bytes * gs_reps
    gs_gbs = gs_bytes / (gs_ms / 1e3) / 1e9
    traffic = gs_traffic(w.name)
    # the same kernel inside the profiled solve (event-bracketed launches)
    gs0 = [p for p in prof if p["name"] == "gs_colour_phase" and p["level"] == 0
           and p["prec"] == hpg.HPG_FP32]
    gs_in_solve = (gs0[0]["bytes"] / (gs0[0]["total_ms"] / 1e3) / 1e9) if gs0 else None
    # whole solve: the library's algorithmic bytes of every launch of one
    # solve (its per-launch byte model, summed by the profiler) over the
    # graph-timed time per solve
    solve_bytes = sum(p["bytes"] for p in prof)
    solve_gbs = solve_bytes / (ms_max / args.steps / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "gs_phase_kernel (level 0, fp32)",
                "achieved": gs_gbs, "peak": peak, "unit": "GB/s", "frac": gs_gbs / peak,
                "peak_source": peak_src,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": gs_bytes / (gs_reps * gs_phases),
                "row_bytes": gs_row_bytes,
                "launches": gs_reps * gs_phases,
                "avg_launch_us": 1e3 * gs_ms / (gs_reps * gs_phases),
                "timing": "CUDA events around each of %d graph-launched hpg_mg_smooth sweeps "
                          "on level 0 (%d phase launches), a graph-launched level-0 SpMV "
                          "between sweeps" % (gs_reps, gs_reps * gs_phases),
                "in_solve": {"achieved": gs_in_solve,
                             "frac": gs_in_solve / peak if gs_in_solve else None,
                             "timing": "level-0 phases of one eager solve, each bracketed "
                                       "by events (launch gaps included)"},
                "solve": {"bytes": solve_bytes, "achieved": solve_gbs,
                          "frac": solve_gbs / peak,
                          "timing": "sum of per-launch algorithmic bytes of one solve over "
                                    "the graph-timed ms_per_step"}}
    kernels = [{"name": p["name"], "level": p["level"], "prec": p["prec"],
                "launches": p["launches"], "share": p["total_ms"] / tot_ms,
                "avg_us": 1e3 * p["total_ms"] / p["launches"],
                "gbs": (p["bytes"] / (p["total_ms"] / 1e3) / 1e9) if p["total_ms"] > 0 else 0}
               for p in prof[:6]]

    # ---- end to end through the C ABI with pinned host buffers
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    for _ in range(1):
        xh.zero_()
        hpg.gmres_ir_solve(prob.h, bh, xh, tol=w.tol, restart=w.restart, maxit=w.maxit,
                           inner=hpg.HPG_FP32, basis=basis_mxp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_fl = 0
    for _ in range(args.steps):
        xh.zero_()
        inf = hpg.gmres_ir_solve(prob.h, bh, xh, tol=w.tol, restart=w.restart, maxit=w.maxit,
                                 inner=hpg.HPG_FP32, basis=basis_mxp)
        e2e_fl += metrics.solve_flops(dims_list, metrics.cycles_from_info(
            inf["iterations"], inf["restarts"], w.restart))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s_max, e2e_fl_sum = reduce_max_sum([e2e_s, e2e_fl], ["max", "sum"], dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample(args.workload, args.cpu_sample_iters)
        cpu = {"value": r["flops"] / r["seconds"] / 1e9, "unit": "GFLOP/s", "cores": 1,
               "kind": "oracle",
               "sample": "%d inner GMRES steps of %s (FP64 numpy/scipy oracle, 1 thread, "
                         "%.1f s; hierarchy build untimed)" % (r["iterations"], w.name,
                                                                 r["seconds"])}
        # context: the same sample with every host core available to BLAS (the
        # sparse products stay single-threaded), and the whole 16^3 FP64 solve
        ra = oracle_sample(args.workload, args.cpu_sample_iters, threads=None)
        r16 = oracle_sample("fp64_gmres30_16cube", 10000)
        cpu["all_cores"] = {"value": ra["flops"] / ra["seconds"] / 1e9,
                            "cores": os.cpu_count(), "seconds": ra["seconds"]}
        cpu["full_solve_16cube"] = {"seconds": r16["seconds"],
                                    "iterations": r16["iterations"],
                                    "value": r16["flops"] / r16["seconds"] / 1e9}

    if rank == 0:
        line = {
            "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.dims), "beta": w.beta,
                       "restart": w.restart, "tol": w.tol, "levels": len(dims_list),
                       "smoother": "1+1 symmetric multicolour Gauss-Seidel",
                       "rhs": "A*1 + N(0, %g^2), seed %d" % (w.noise_std, w.seed),
                       "inner": "fp32", "basis": args.basis, "outer": "fp64",
                       "l2": "inputs larger than L2 (FP32 ELL matrix %.0f MB)" % (
                           prob.n_store() * 27 * 8 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": launches, "clocks": clocks,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_fl_sum / e2e_s_max / 1e9, "unit": "GFLOP/s",
                    "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n},
            "kernels": kernels,
            "validation": valid,
            "penalized_value": gflops * valid["penalty"] if valid else None,
            "iterations": n_ir, "rel_residual": infos[-1]["rel_residual"],
            "roofline": roofline,
            "time_to_solution_ms": ms_max / args.steps,
            "fp64": fp64,
            "speedup_vs_fp64": (gflops / fp64["value"]) if fp64 else None,
            "time_speedup_vs_fp64": (fp64["ms_per_solve"] / (ms_max / args.steps)) if fp64
            else None,
        }
        line = rounded(line)
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
