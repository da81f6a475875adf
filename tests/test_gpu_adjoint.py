"""Differentiable solve (paper_2507_11512_gb300.adjoint): gradients through the
library's GMRES-IR against the oracle's dense adjoint and against central
finite differences of the GPU solve itself."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from oracle import hpg_oracle as O  # noqa: E402
from paper_2507_11512_gb300 import adjoint  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def inputs(dims, seed):
    n = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.9, 1.1, n)
    b = rng.standard_normal(n)
    xt = rng.standard_normal(n)
    return theta, b, xt


def gpu_grads(dims, beta, theta, b, xt, **kw):
    bt = torch.tensor(b, device=DEV, requires_grad=True)
    tt = torch.tensor(theta, device=DEV, requires_grad=True)
    x = adjoint.solve(bt, tt, dims, beta, **kw)
    loss = ((x - torch.tensor(xt, device=DEV)) ** 2).sum()
    loss.backward()
    return (x.detach().cpu().numpy(), loss.item(), bt.grad.cpu().numpy(),
            tt.grad.cpu().numpy())


@pytest.mark.parametrize("inner", [hpg.HPG_FP32, hpg.HPG_FP64])
@pytest.mark.parametrize("beta", [0.5, 0.0])
def test_gradients_match_oracle_dense_adjoint(inner, beta):
    dims = (12, 12, 12)
    theta, b, xt = inputs(dims, 11)
    x_o, L_o, gb_o, gt_o = O.dense_adjoint_gradients(*dims, b, xt, beta, theta)
    x, L, gb, gt = gpu_grads(dims, beta, theta, b, xt, tol=1e-12, inner=inner)
    assert np.linalg.norm(x - x_o) <= 1e-9 * np.linalg.norm(x_o)
    assert abs(L - L_o) <= 1e-9 * L_o
    assert np.linalg.norm(gb - gb_o) <= 1e-8 * np.linalg.norm(gb_o)
    assert np.linalg.norm(gt - gt_o) <= 1e-8 * np.linalg.norm(gt_o)


def test_gradients_match_central_differences_of_the_gpu_solve():
    dims, beta, h = (12, 12, 12), 0.5, 1e-6
    theta, b, xt = inputs(dims, 12)
    _, _, gb, gt = gpu_grads(dims, beta, theta, b, xt, tol=1e-13, inner=hpg.HPG_FP64)
    xtt = torch.tensor(xt, device=DEV)

    def loss(bv, tv):
        with torch.no_grad():
            x = adjoint.solve(torch.tensor(bv, device=DEV), torch.tensor(tv, device=DEV), dims,
                              beta, tol=1e-13, inner=hpg.HPG_FP64)
            return ((x - xtt) ** 2).sum().item()

    rng = np.random.default_rng(0)
    for i in rng.choice(b.size, 4, replace=False):
        e = np.zeros(b.size)
        e[i] = h
        fd_b = (loss(b + e, theta) - loss(b - e, theta)) / (2 * h)
        fd_t = (loss(b, theta + e) - loss(b, theta - e)) / (2 * h)
        assert abs(fd_b - gb[i]) <= 1e-5 * np.abs(gb).max()
        assert abs(fd_t - gt[i]) <= 1e-5 * np.abs(gt).max()


def test_low_precision_basis_gradients():
    dims, beta = (12, 12, 12), 0.5
    theta, b, xt = inputs(dims, 13)
    _, _, gb_o, gt_o = O.dense_adjoint_gradients(*dims, b, xt, beta, theta)
    _, _, gb, gt = gpu_grads(dims, beta, theta, b, xt, tol=1e-12, basis=hpg.HPG_BF16)
    assert np.linalg.norm(gb - gb_o) <= 1e-8 * np.linalg.norm(gb_o)
    assert np.linalg.norm(gt - gt_o) <= 1e-8 * np.linalg.norm(gt_o)


def test_only_requested_gradients_and_zero_cotangent():
    dims = (8, 8, 8)
    theta, b, xt = inputs(dims, 14)
    bt = torch.tensor(b, device=DEV)
    tt = torch.tensor(theta, device=DEV, requires_grad=True)
    x = adjoint.solve(bt, tt, dims, 0.5)
    (0.0 * x.sum()).backward()
    assert bt.grad is None and torch.count_nonzero(tt.grad) == 0


def test_96cube_forward_and_adjoint_residuals():
    """The differentiable-solve workload size: both solves reach the tolerance
    (checked with the library's FP64 SpMV on the same operators)."""
    dims, beta = (96, 96, 96), 0.5
    n = 96 ** 3
    g = torch.Generator(device="cpu").manual_seed(0)
    theta = (0.9 + 0.2 * torch.rand(n, generator=g, dtype=torch.float64)).to(DEV)
    b = torch.randn(n, generator=g, dtype=torch.float64).to(DEV)
    xt = torch.randn(n, generator=g, dtype=torch.float64).to(DEV)
    bt = b.clone().requires_grad_(True)
    tt = theta.clone().requires_grad_(True)
    x = adjoint.solve(bt, tt, dims, beta, tol=1e-9)
    loss = ((x - xt) ** 2).sum()
    loss.backward()
    lam = bt.grad
    for sgn, rhs, sol in [(1, b, x.detach()), (-1, 2 * (x.detach() - xt), lam)]:
        with hpg.Problem(*dims, beta=sgn * beta, theta=theta) as p:
            ax = p.to_natural(p.spmv(p.to_storage(sol)))
        assert torch.linalg.norm(rhs - ax) <= 1e-9 * torch.linalg.norm(rhs)
    assert torch.allclose(tt.grad, -26.0 * lam * x.detach(), rtol=0, atol=0)


def test_diag_scale_gradient_kernel_and_problem_reuse():
    """hpg_diag_scale_gradient computes (-26 lambda_i) x_i; repeated passes
    with the same theta reuse the cached forward and adjoint problems, and a
    new theta builds new ones."""
    dims = (16, 12, 8)
    n = 16 * 12 * 8
    theta, b, xt = inputs(dims, 15)
    adjoint.clear_cache()
    s0 = adjoint.cache_stats()
    g1 = gpu_grads(dims, 0.5, theta, b, xt, tol=1e-12)
    g2 = gpu_grads(dims, 0.5, theta, b, xt, tol=1e-12)
    s1 = adjoint.cache_stats()
    assert s1["builds"] - s0["builds"] == 2 and s1["reuses"] - s0["reuses"] == 2
    for a, c in zip(g1[2:], g2[2:]):
        np.testing.assert_array_equal(a, c)
    gpu_grads(dims, 0.5, theta * 1.01, b, xt, tol=1e-12)
    assert adjoint.cache_stats()["builds"] - s1["builds"] == 2
    adjoint.clear_cache()
    rng = np.random.default_rng(2)
    lam = torch.tensor(rng.standard_normal(n), device=DEV)
    x = torch.tensor(rng.standard_normal(n), device=DEV)
    out = torch.full_like(x, float("nan"))
    with hpg.Problem(*dims, beta=0.5, theta=theta) as p:
        hpg.diag_scale_gradient(p.h, lam, x, out)
        torch.testing.assert_close(out, (-26.0 * lam) * x, rtol=0, atol=0)
        with pytest.raises(hpg.HpgError):
            hpg.diag_scale_gradient(p.h, lam, None, out)
