"""Command-line solve driver: sets up a synthetic HPG-MxP problem and runs
GMRES-IR solves through the C ABI, printing one JSON line per solve.

  python -m paper_2507_11512_gb300.runsolve --grid 128 128 128 --inner fp32 \\
      --solves 2 --warmup 1 [--maxit N] [--profile] [--option GS_HALO=1] \\
      [--sweeps 20]

The right-hand side is b = A*1 + N(0, noise^2) (seeded); x0 = 0.  Intended
for profiling runs (ncu, the built-in event profiler), A/B timing of the
implementation options (hpg_set_option) and quick checks.  Every solve line
carries its CUDA-event time (`event_ms`); --sweeps K also times K
graph-launched level-0 symmetric Gauss-Seidel sweeps (hpg_mg_smooth, inner
precision), each after a graph-launched level-0 SpMV as in the solve.
"""

import argparse
import json
import time

import torch

import paper_2507_11512_gb300 as hpg


def time_sweeps(p, reps, dtype):
    """CUDA-event time of `reps` graph-launched symmetric sweeps on level 0
    (15 colour phases each), a graph-launched level-0 SpMV before each."""
    dev = torch.device("cuda", torch.cuda.current_device())
    n = p.info[0]["n"]
    g = torch.Generator(device=dev).manual_seed(1)
    r = p.to_storage(torch.randn(n, dtype=torch.float64, device=dev, generator=g), dtype=dtype)
    z = torch.zeros_like(r)
    w = torch.empty_like(r)
    hpg.mg_smooth(p.h, 0, r, z, 1, False)
    torch.cuda.synchronize()
    g_spmv, g_sweep = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_spmv):
        hpg.spmv(p.h, 0, r, w)
    with torch.cuda.graph(g_sweep):
        hpg.mg_smooth(p.h, 0, r, z, 1, False)
    for _ in range(3):
        g_spmv.replay()
        g_sweep.replay()
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for e0, e1 in ev:
        g_spmv.replay()
        e0.record(st)
        g_sweep.replay()
        e1.record(st)
    torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    return {"sweeps": reps, "sweep_us": 1e3 * ms / reps, "phase_us": 1e3 * ms / (15 * reps)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=3, default=[128, 128, 128])
    ap.add_argument("--beta", type=float, default=0.5)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--maxit", type=int, default=10000)
    ap.add_argument("--inner", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--basis", choices=["same", "bf16", "fp16"], default="same")
    ap.add_argument("--noise", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--eager", action="store_true",
                    help="host-driven solve (kernels visible to ncu one by one)")
    ap.add_argument("--profile", action="store_true",
                    help="host-driven solve with per-kernel CUDA-event timing")
    ap.add_argument("--option", action="append", default=[],
                    help="NAME=VALUE for hpg_set_option (e.g. GS_HALO=1, PDL=0)")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="time this many graph-launched level-0 sweeps after the solves")
    a = ap.parse_args(argv)
    from paper_2507_11512_gb300 import build
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    inner = hpg.HPG_FP32 if a.inner == "fp32" else hpg.HPG_FP64
    basis = {"same": inner, "bf16": hpg.HPG_BF16, "fp16": hpg.HPG_FP16}[a.basis]
    with hpg.Problem(*a.grid, beta=a.beta, levels=a.levels) as p:
        n = a.grid[0] * a.grid[1] * a.grid[2]
        ones = torch.ones(n, dtype=torch.float64, device=dev)
        b = p.to_natural(p.spmv(p.to_storage(ones)))
        g = torch.Generator(device="cpu").manual_seed(a.seed)
        b += a.noise * torch.randn(n, generator=g, dtype=torch.float64).to(dev)
        x = torch.zeros_like(b)
        for o in a.option:
            name, val = o.split("=")
            hpg.set_option(p.h, getattr(hpg, "HPG_OPT_" + name.upper()), int(val))
        if a.eager:
            hpg.set_execution(p.h, hpg.HPG_EXEC_EAGER)
        for _ in range(a.warmup):
            x.zero_()
            hpg.gmres_ir_solve(p.h, b, x, tol=a.tol, restart=a.restart, maxit=a.maxit,
                               inner=inner, basis=basis)
        if a.profile:
            hpg.set_profiling(p.h, True)
        st = torch.cuda.current_stream()
        for _ in range(a.solves):
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(st)
            info = hpg.gmres_ir_solve(p.h, b, x, tol=a.tol, restart=a.restart, maxit=a.maxit,
                                      inner=inner, basis=basis)
            e1.record(st)
            torch.cuda.synchronize()
            info["ms"] = 1e3 * (time.perf_counter() - t0)
            info["event_ms"] = e0.elapsed_time(e1)
            print(json.dumps(info), flush=True)
        if a.sweeps > 0:
            print(json.dumps(time_sweeps(p, a.sweeps, torch.float32 if a.inner == "fp32"
                                         else torch.float64)), flush=True)
        if a.profile:
            rep = hpg.profile_report(p.h)
            rep.sort(key=lambda r: -r["total_ms"])
            for r in rep:
                r["avg_us"] = 1e3 * r["total_ms"] / max(1, r["launches"])
                r["gbs"] = r["bytes"] / max(1e-12, r["total_ms"] * 1e-3) / 1e9
                print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
