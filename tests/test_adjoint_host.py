"""Host-side checks of the differentiable solve's wrapper (no GPU needed):
arguments are validated before anything reaches the library, and the
gradient formula of the backward pass is the adjoint one (checked on a dense
CPU stand-in for the solve)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_11512_gb300 import adjoint  # noqa: E402


def test_rejects_wrong_sizes_and_dtypes():
    dims = (4, 4, 4)
    n = 64
    b = torch.zeros(n, dtype=torch.float64)
    theta = torch.ones(n, dtype=torch.float64)
    with pytest.raises(ValueError):
        adjoint.solve(b[:-1], theta, dims)
    with pytest.raises(ValueError):
        adjoint.solve(b, theta[:-1], dims)
    with pytest.raises(TypeError):
        adjoint.solve(b.float(), theta, dims)
    with pytest.raises(TypeError):
        adjoint.solve(b, theta.float(), dims)


def test_backward_is_the_adjoint_formula(monkeypatch):
    """With the library replaced by dense CPU stand-ins of the same operator
    (the oracle's matrix; the gradient call as its header states it),
    autograd through StencilSolve gives dL/db = A^{-T} g and dL/dtheta_i =
    -26 lambda_i x_i, which central differences confirm: the wrapper solves
    the adjoint on A(-beta) and passes lambda and x in the right order."""
    from oracle import hpg_oracle as O
    dims, beta = (3, 3, 2), 0.5
    n = 18

    class FakeProblem:
        def __init__(self, dims_, beta_, theta, levels):
            self.h = (tuple(dims_), beta_, theta.clone())

    def dense_solve(p, beta_, rhs, tol, restart, maxit, inner, basis):
        dims_, b_, theta = p.h
        assert b_ == beta_
        A = O.build_matrix(*dims_, b_, theta.numpy()).toarray()
        x = np.linalg.solve(A, rhs.numpy())
        return torch.tensor(x, dtype=torch.float64), {"status": 0}

    def gradient(h, lam, x, grad, stream=None):
        grad.copy_((-26.0 * lam) * x)

    monkeypatch.setattr(adjoint, "_problem", FakeProblem)
    monkeypatch.setattr(adjoint, "_solve", dense_solve)
    monkeypatch.setattr(adjoint, "diag_scale_gradient", gradient)
    rng = np.random.default_rng(0)
    theta0 = torch.tensor(rng.uniform(0.9, 1.1, n))
    b0 = torch.tensor(rng.standard_normal(n))
    xt = torch.tensor(rng.standard_normal(n))

    def loss(b, theta):
        x = adjoint.solve(b, theta, dims, beta)
        return ((x - xt) ** 2).sum()

    b = b0.clone().requires_grad_(True)
    theta = theta0.clone().requires_grad_(True)
    loss(b, theta).backward()
    h = 1e-6
    for i in (0, 7, 17):
        e = torch.zeros(n, dtype=torch.float64)
        e[i] = h
        fd_b = (loss(b0 + e, theta0) - loss(b0 - e, theta0)).item() / (2 * h)
        fd_t = (loss(b0, theta0 + e) - loss(b0, theta0 - e)).item() / (2 * h)
        assert abs(b.grad[i].item() - fd_b) <= 1e-6 * max(1.0, abs(fd_b))
        assert abs(theta.grad[i].item() - fd_t) <= 1e-6 * max(1.0, abs(fd_t))
