"""Differentiable GMRES-IR solve: x = A(theta)^{-1} b as a torch.autograd.Function.

Forward runs the library's mixed-precision GMRES-IR on A(theta) (the 27-point
stencil with diagonal 26 * theta_i, nonsymmetric option beta).  Backward is the
adjoint: it solves A(theta)^T lambda = dL/dx with the same solver on the
transposed operator, which is the same stencil with beta -> -beta and the same
diagonal, and returns

    dL/db = lambda,      dL/dtheta_i = -lambda_i * 26 * x_i

(only a_ii = 26 theta_i depends on theta_i).  Both solves run entirely in the
library's CUDA kernels; this module only builds the two problems and moves
tensors.  Vectors are FP64 in natural order on the GPU.
"""

import torch

from . import HPG_FP32, HpgError, Problem, gmres_ir_solve

DIAG = 26.0


def _solve(dims, beta, theta, rhs, tol, restart, maxit, inner, basis, levels):
    with Problem(*dims, beta=beta, theta=theta, levels=levels) as p:
        x = torch.zeros_like(rhs)
        info = gmres_ir_solve(p.h, rhs.contiguous(), x, tol=tol, restart=restart, maxit=maxit,
                              inner=inner, basis=basis)
    if info["status"] != 0:
        raise HpgError(info["status"], "differentiable solve (beta %g)" % beta)
    return x, info


class StencilSolve(torch.autograd.Function):
    """x = A(theta)^{-1} b; gradients for b and theta by the adjoint solve."""

    @staticmethod
    def forward(ctx, b, theta, dims, beta, tol, restart, maxit, inner, basis, levels):
        x, info = _solve(dims, beta, theta.detach(), b.detach(), tol, restart, maxit, inner,
                         basis, levels)
        ctx.save_for_backward(theta, x)
        ctx.cfg = (dims, beta, tol, restart, maxit, inner, basis, levels)
        ctx.forward_info = info
        return x

    @staticmethod
    def backward(ctx, g):
        theta, x = ctx.saved_tensors
        dims, beta, tol, restart, maxit, inner, basis, levels = ctx.cfg
        if not torch.any(g != 0):
            lam = torch.zeros_like(g)
        else:
            lam, _ = _solve(dims, -beta, theta.detach(), g.detach().to(torch.float64), tol,
                            restart, maxit, inner, basis, levels)
        grad_b = lam if ctx.needs_input_grad[0] else None
        grad_theta = (-DIAG) * lam * x if ctx.needs_input_grad[1] else None
        return grad_b, grad_theta, None, None, None, None, None, None, None, None


def solve(b, theta, dims, beta=0.0, tol=1e-10, restart=30, maxit=10000, inner=HPG_FP32,
          basis=None, levels=4):
    """Differentiable x = A(theta)^{-1} b.  b, theta: FP64 CUDA tensors of
    nx*ny*nz entries in natural order (either may require grad)."""
    if basis is None:
        basis = inner
    n = dims[0] * dims[1] * dims[2]
    if b.numel() != n or theta.numel() != n:
        raise ValueError("b and theta need %d entries" % n)
    if b.dtype != torch.float64 or theta.dtype != torch.float64:
        raise TypeError("b and theta must be float64")
    return StencilSolve.apply(b, theta, tuple(dims), float(beta), tol, restart, maxit, inner,
                              basis, levels)


def main(argv=None):
    """Times forward + adjoint on the differentiable-solve workload:
    python -m paper_2507_11512_gb300.adjoint [--grid 96 96 96] [--reps 3]
    theta ~ U(0.9, 1.1), b ~ N(0, 1), x_target ~ N(0, 1) (seed 0, host
    generator), beta 0.5, L = ||x - x_target||^2.  Prints one JSON line."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=3, default=[96, 96, 96])
    ap.add_argument("--beta", type=float, default=0.5)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    dims = tuple(a.grid)
    n = dims[0] * dims[1] * dims[2]
    dev = torch.device("cuda")
    g = torch.Generator(device="cpu").manual_seed(0)
    theta = (0.9 + 0.2 * torch.rand(n, generator=g, dtype=torch.float64)).to(dev)
    b = torch.randn(n, generator=g, dtype=torch.float64).to(dev)
    xt = torch.randn(n, generator=g, dtype=torch.float64).to(dev)
    times = []
    for it in range(a.reps + 1):
        bt = b.clone().requires_grad_(True)
        tt = theta.clone().requires_grad_(True)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        x = solve(bt, tt, dims, a.beta, tol=a.tol)
        loss = ((x - xt) ** 2).sum()
        e1.record()
        loss.backward()
        e2.record()
        torch.cuda.synchronize()
        if it > 0:
            times.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    fwd = sorted(t[0] for t in times)[len(times) // 2]
    bwd = sorted(t[1] for t in times)[len(times) // 2]
    print(json.dumps({"workload": "diff_solve_%dx%dx%d" % dims, "beta": a.beta, "tol": a.tol,
                      "forward_ms": fwd, "backward_ms": bwd, "loss": loss.item(),
                      "grad_theta_norm": tt.grad.norm().item(),
                      "note": "each pass builds its problem (matrix + hierarchy) and solves"}))


if __name__ == "__main__":
    main()
