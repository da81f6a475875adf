"""Full-size checks at the benchmark sizes (128^3 GMRES(30), 320^3 GMRES(50)),
in the launch configuration the bench times: SpMV on sampled rows against
the oracle's row-by-row definition, the smoother's last colour phase against
its defining equation, V-cycle linearity, and the solves' FP64 residual
recomputed with the separately checked FP64 SpMV."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from oracle import hpg_oracle as O  # noqa: E402
from tests.gpu_helpers import FP32_ELEM  # noqa: E402
from workloads import WORKLOADS, rhs_noise  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
SIZES = [("mxp_gmres30_128cube", 128), ("mxp_gmres50_320cube", 320)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def sample_points(N, count, seed):
    rng = np.random.default_rng(seed)
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(count)]
    # corners, faces and the last point: the truncated boundary rows
    pts += [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N // 2, N - 1), (N - 1, 0, N // 3),
            (N // 2, N // 2, 0), (N - 1, N - 1, 0)]
    return pts


@pytest.mark.parametrize("name,N", SIZES)
def test_spmv_sampled_rows_full_size(name, N):
    beta = WORKLOADS[name].beta
    n = N ** 3
    g = torch.Generator(device="cpu").manual_seed(7)
    x64 = torch.randn(n, generator=g, dtype=torch.float64)
    x32 = x64.to(torch.float32)
    with hpg.Problem(N, N, N, beta=beta) as p:
        y64 = p.to_natural(p.spmv(p.to_storage(x64.to(DEV)))).cpu().numpy()
        y32 = p.to_natural(p.spmv(p.to_storage(x32.to(DEV)))).cpu().numpy()
    xn, xf = x64.numpy(), x32.numpy().astype(np.float64)
    for (i, j, k) in sample_points(N, 400, 1):
        row = O.stencil_row(N, N, N, i, j, k, beta)
        q = O.natural_index(i, j, k, N, N)
        ref = sum(v * xn[c] for c, v in row)
        mag = sum(abs(v * xn[c]) for c, v in row)
        assert abs(y64[q] - ref) <= 1e-13 * mag
        ref32 = sum(v * xf[c] for c, v in row)
        mag32 = sum(abs(v * xf[c]) for c, v in row)
        assert abs(float(y32[q]) - ref32) <= FP32_ELEM * mag32


@pytest.mark.parametrize("name,N", SIZES)
def test_last_colour_of_a_sweep_full_size(name, N):
    """After a symmetric sweep the last phase (colour 0 of the backward half)
    saw every neighbour at its final value, so each colour-0 point satisfies
    z_i = (r_i - sum_j a_ij z_j) / a_ii with the returned z."""
    beta = WORKLOADS[name].beta
    n = N ** 3
    g = torch.Generator(device="cpu").manual_seed(8)
    r_nat = torch.randn(n, generator=g, dtype=torch.float64).to(torch.float32)
    with hpg.Problem(N, N, N, beta=beta) as p:
        r_st = p.to_storage(r_nat.to(DEV))
        z_st = torch.zeros_like(r_st)
        hpg.mg_smooth(p.h, 0, r_st, z_st, 1, True)
        z = p.to_natural(z_st).cpu().numpy().astype(np.float64)
    rn = r_nat.numpy().astype(np.float64)
    checked = 0
    for (i, j, k) in sample_points(N, 3000, 2):
        if O.colour_of(i, j, k) != 0:
            continue
        row = O.stencil_row(N, N, N, i, j, k, beta)
        q = O.natural_index(i, j, k, N, N)
        off = sum(v * z[c] for c, v in row if c != q)
        mag = abs(rn[q]) + sum(abs(v * z[c]) for c, v in row if c != q)
        assert abs(z[q] * 26.0 - (rn[q] - off)) <= FP32_ELEM * mag * 2
        checked += 1
    assert checked > 200


@pytest.mark.parametrize("name,N", SIZES)
def test_vcycle_linear_full_size(name, N):
    beta = WORKLOADS[name].beta
    with hpg.Problem(N, N, N, beta=beta) as p:
        ns = p.n_store()
        g = torch.Generator(device="cpu").manual_seed(9)
        mask = p.to_storage(torch.ones(N ** 3, dtype=torch.float32, device=DEV)) != 0
        r1 = torch.where(mask, torch.randn(ns, generator=g).to(DEV), torch.zeros(ns, device=DEV))
        r2 = torch.where(mask, torch.randn(ns, generator=g).to(DEV), torch.zeros(ns, device=DEV))
        z1, z2, z12 = p.vcycle(r1), p.vcycle(r2), p.vcycle(r1 + r2)
    err = torch.linalg.norm((z12 - z1 - z2).double())
    # three FP32 V-cycles, each within the 1e-6 FP32 V-cycle tolerance
    assert err <= 3e-6 * torch.linalg.norm((z1 + z2).double())


@pytest.mark.parametrize("name,N", SIZES)
def test_solve_full_size_residual(name, N):
    w = WORKLOADS[name]
    n = N ** 3
    with hpg.Problem(N, N, N, beta=w.beta) as p:
        ones = torch.ones(n, dtype=torch.float64, device=DEV)
        b = p.to_natural(p.spmv(p.to_storage(ones)))
        b += torch.tensor(rhs_noise(n, w.noise_std, w.seed), device=DEV)
        x = torch.zeros_like(b)
        info = hpg.gmres_ir_solve(p.h, b, x, tol=w.tol, restart=w.restart, maxit=w.maxit,
                                  inner=hpg.HPG_FP32)
        assert info["status"] == 0 and info["converged"] == 1
        ax = p.to_natural(p.spmv(p.to_storage(x)))
        rel = (torch.linalg.norm(b - ax) / torch.linalg.norm(b)).item()
    assert rel < w.tol
    assert abs(rel - info["rel_residual"]) <= 1e-3 * w.tol
