"""Low-precision Krylov basis (BF16 / FP16 with one FP32 scale per vector)
inside the FP64 refinement: the refined solution matches the oracle's, the
graph and host-driven solves agree bitwise, and the per-vector scaling keeps
FP16 safe for right-hand sides of any magnitude."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from oracle import hpg_oracle as O  # noqa: E402
from tests.gpu_helpers import oracle_hierarchy  # noqa: E402
from workloads import rhs_noise, x_true  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
BASES = [hpg.HPG_BF16, hpg.HPG_FP16]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def solve(dims, beta, b, basis, tol=1e-12, restart=30, maxit=10000, eager=False):
    with hpg.Problem(*dims, beta=beta, levels=4) as p:
        if eager:
            hpg.set_execution(p.h, hpg.HPG_EXEC_EAGER)
        bt = torch.tensor(b, dtype=torch.float64, device=DEV)
        xt = torch.zeros_like(bt)
        info = hpg.gmres_ir_solve(p.h, bt, xt, tol=tol, restart=restart, maxit=maxit,
                                  inner=hpg.HPG_FP32, basis=basis)
        return xt.cpu().numpy(), info


@pytest.mark.parametrize("basis", BASES)
@pytest.mark.parametrize("dims,beta", [((16, 16, 16), 0.5), ((24, 20, 28), 0.0)])
def test_low_precision_basis_matches_oracle(basis, dims, beta):
    lv = oracle_hierarchy(dims, 4, beta)
    n = lv[0].n
    b = lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=0)
    x_o, info_o = O.gmres_ir(lv, b, tol=1e-12, restart=30)
    x, info = solve(dims, beta, b, basis)
    assert info["status"] == 0 and info["converged"] == 1
    r = np.linalg.norm(b - lv[0].A @ x) / np.linalg.norm(b)
    assert r < 1e-12
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= 1e-8
    # a 2-byte basis costs extra inner steps, not convergence
    assert info["iterations"] <= 3 * info_o.iterations + 10


@pytest.mark.parametrize("basis", BASES)
def test_low_precision_basis_restart50(basis):
    # restart 50 takes the 64-column CGS2 instantiation
    dims, beta = (16, 16, 16), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    b = lv[0].A @ x_true(lv[0].n)
    x, info = solve(dims, beta, b, basis, tol=1e-10, restart=50)
    assert info["status"] == 0
    assert np.linalg.norm(b - lv[0].A @ x) / np.linalg.norm(b) < 1e-10
    assert np.abs(x - 1.0).max() < 1e-7


@pytest.mark.parametrize("basis", BASES)
def test_graph_and_eager_agree_bitwise(basis):
    dims = (16, 16, 16)
    lv = oracle_hierarchy(dims, 4, 0.5)
    b = lv[0].A @ x_true(lv[0].n) + rhs_noise(lv[0].n, 1e-3, seed=1)
    xg, ig = solve(dims, 0.5, b, basis, tol=1e-10)
    xe, ie = solve(dims, 0.5, b, basis, tol=1e-10, eager=True)
    assert ig["graph_launches"] == 1 and ie["graph_launches"] == 0
    assert ig["iterations"] == ie["iterations"]
    assert np.array_equal(xg, xe)


@pytest.mark.parametrize("scale", [1e30, 1e-30])
def test_fp16_basis_any_rhs_magnitude(scale):
    # q_j is stored as q_j / max|q_j|: the FP16 range never limits the basis
    dims, beta = (12, 12, 12), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    b0 = lv[0].A @ x_true(lv[0].n)
    x, info = solve(dims, beta, scale * b0, hpg.HPG_FP16, tol=1e-10)
    assert info["status"] == 0 and info["converged"] == 1
    assert np.abs(x / scale - 1.0).max() < 1e-7


def test_unsupported_basis_combinations():
    with hpg.Problem(8, 8, 8) as p:
        b = torch.ones(512, dtype=torch.float64, device=DEV)
        x = torch.zeros_like(b)
        for inner, basis in [(hpg.HPG_FP64, hpg.HPG_BF16), (hpg.HPG_FP64, hpg.HPG_FP32),
                             (hpg.HPG_BF16, hpg.HPG_BF16), (hpg.HPG_FP32, hpg.HPG_FP64)]:
            with pytest.raises(hpg.HpgError):
                hpg.gmres_ir_solve(p.h, b, x, inner=inner, basis=basis)


def test_deterministic_bitwise_bf16():
    dims = (16, 16, 16)
    lv = oracle_hierarchy(dims, 4, 0.5)
    b = lv[0].A @ x_true(lv[0].n) + rhs_noise(lv[0].n, 1e-3, seed=2)
    x1, i1 = solve(dims, 0.5, b, hpg.HPG_BF16, tol=1e-10)
    x2, i2 = solve(dims, 0.5, b, hpg.HPG_BF16, tol=1e-10)
    assert i1["iterations"] == i2["iterations"] and np.array_equal(x1, x2)
