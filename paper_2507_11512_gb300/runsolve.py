"""Command-line solve driver: sets up a synthetic HPG-MxP problem and runs
GMRES-IR solves through the C ABI, printing one JSON line per solve.

  python -m paper_2507_11512_gb300.runsolve --grid 128 128 128 --inner fp32 \\
      --solves 2 --warmup 1 [--maxit N] [--profile]

The right-hand side is b = A*1 + N(0, noise^2) (seeded); x0 = 0.  Intended
for profiling runs (ncu, the built-in event profiler) and quick checks.
"""

import argparse
import json
import time

import torch

import paper_2507_11512_gb300 as hpg


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
        if a.eager:
            hpg.set_execution(p.h, hpg.HPG_EXEC_EAGER)
        for _ in range(a.warmup):
            x.zero_()
            hpg.gmres_ir_solve(p.h, b, x, tol=a.tol, restart=a.restart, maxit=a.maxit,
                               inner=inner, basis=basis)
        if a.profile:
            hpg.set_profiling(p.h, True)
        for _ in range(a.solves):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = hpg.gmres_ir_solve(p.h, b, x, tol=a.tol, restart=a.restart, maxit=a.maxit,
                                      inner=inner, basis=basis)
            info["ms"] = 1e3 * (time.perf_counter() - t0)
            print(json.dumps(info), flush=True)
        if a.profile:
            rep = hpg.profile_report(p.h)
            rep.sort(key=lambda r: -r["total_ms"])
            for r in rep:
                r["avg_us"] = 1e3 * r["total_ms"] / max(1, r["launches"])
                r["gbs"] = r["bytes"] / max(1e-12, r["total_ms"] * 1e-3) / 1e9
                print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
