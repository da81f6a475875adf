"""Oracle parity at the sizes whose matrices stream from HBM.

On a level whose FP32 ELL arrays (27 slots x (4-byte value + 4-byte index)
per storage row) exceed 96 MiB, the library runs its bandwidth kernels:
the streamed Gauss-Seidel colour phase (every slot, and the first forward
sweep's per-colour slot sets), the phases that keep their matrix slice in L2
(colour 6 forward, colour 0 last, where a slice fits in 96 MiB), and the
streamed fused residual-restriction.  The small-grid parity tests never reach
those kernels, so these tests compare them with the FP64 oracle element by
element at grids from 80^3 to 160^3, in the launch configuration of the
128^3 benchmark solve:

* hpg_mg_smooth (eqs. (1)-(2), Sec. 3.2.1): 1 and 2 sweeps from z = 0 and one
  from a given iterate, against the oracle's colour phases;
* hpg_mg_vcycle (Fig. 1, Sec. 3.2.4) from every level, against the oracle's
  V-cycle;
* GMRES-IR (Algorithm 3) to 1e-12, against the oracle's solution: the kernels
  that write the V-cycle's input (cycle start, Arnoldi scaling, the 2-byte
  basis quantisation) also run the first colour phase of level 0 there.

Tolerances: FP64 1e-13 relative in the max norm, FP32 1e-6 relative in the
2-norm (per smoother or V-cycle call); solves 1e-8 relative after refinement.
FP32 inputs are drawn and rounded before both sides see them.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from oracle import hpg_oracle as O  # noqa: E402
from tests.gpu_helpers import (FP32_REL, FP64_REL, oracle_hierarchy, to_natural,  # noqa: E402
                               to_storage)
from workloads import random_vector, rhs_noise, x_true  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
BETA = 0.5
STREAM_BYTES = 96 << 20   # FP32 ELL bytes above which a level's matrix streams
KEEP_SLICE_BYTES = 96 << 20   # a colour slice kept in L2 must fit in this

# 80^3: smallest cube that streams; 82 x 78 x 84: odd colour-block extents and
# ragged 32-row padding (two levels); 128^3: the benchmark grid; 160^3: level 0
# slices too large to keep (the 320^3 configuration) and level 1 streamed too
GRIDS = [(80, 80, 80), (82, 78, 84), (128, 128, 128), (160, 160, 160)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def streamed(info):
    return info["n_store"] * 27 * 8 > STREAM_BYTES


def max_slice_bytes(info):
    cnt = [info["colour_offset"][c + 1] - info["colour_offset"][c] for c in range(8)]
    return max(cnt) * 27 * 8


def close(z, ref, dtype):
    if dtype == torch.float64:
        return np.abs(z - ref).max() <= FP64_REL * np.abs(ref).max()
    return np.linalg.norm(z - ref) <= FP32_REL * np.linalg.norm(ref)


def npdtype(dtype):
    return np.float64 if dtype == torch.float64 else np.float32


def test_grids_take_the_streamed_branches():
    """The grids above reach the kernels this file is about."""
    seen_keep, seen_nokeep, seen_streamed_coarse = False, False, False
    for dims in GRIDS:
        with hpg.Problem(*dims, beta=BETA) as p:
            assert streamed(p.info[0]), dims
            if max_slice_bytes(p.info[0]) <= KEEP_SLICE_BYTES:
                seen_keep = True
            else:
                seen_nokeep = True
            if p.levels > 1 and streamed(p.info[1]):
                seen_streamed_coarse = True
    assert seen_keep and seen_nokeep and seen_streamed_coarse


@pytest.mark.parametrize("dims", GRIDS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_streamed_smooth_matches_oracle(dims, dtype):
    lv = oracle_hierarchy(dims, 4, BETA)
    with hpg.Problem(*dims, beta=BETA, levels=4) as p:
        for l, L in enumerate(lv):
            if not streamed(p.info[l]):
                continue
            r = random_vector(L.n, seed=61 + l, dtype=npdtype(dtype)).astype(np.float64)
            z0 = random_vector(L.n, seed=71 + l, dtype=npdtype(dtype)).astype(np.float64)
            rt = torch.tensor(to_storage(r, L.dims), dtype=dtype, device=DEV)
            for sweeps, zero in [(1, True), (2, True), (1, False)]:
                if zero:
                    # z enters as 0 and is never read: NaN rows prove it
                    zt = torch.tensor(to_storage(np.full(L.n, np.nan), L.dims), dtype=dtype,
                                      device=DEV)
                    ref = np.zeros(L.n)
                else:
                    zt = torch.tensor(to_storage(z0, L.dims), dtype=dtype, device=DEV)
                    ref = z0.copy()
                hpg.mg_smooth(p.h, l, rt, zt, sweeps, zero)
                for _ in range(sweeps):
                    O.symgs(L, r, ref)
                z = to_natural(zt.cpu().numpy(), L.dims).astype(np.float64)
                assert np.isfinite(z).all()
                assert close(z, ref, dtype), (dims, l, sweeps, zero)


@pytest.mark.parametrize("dims", GRIDS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_streamed_vcycle_matches_oracle(dims, dtype):
    lv = oracle_hierarchy(dims, 4, BETA)
    with hpg.Problem(*dims, beta=BETA, levels=4) as p:
        assert p.levels == len(lv)
        for l, L in enumerate(lv):
            r = random_vector(L.n, seed=81 + l, dtype=npdtype(dtype)).astype(np.float64)
            rt = torch.tensor(to_storage(r, L.dims), dtype=dtype, device=DEV)
            z = to_natural(p.vcycle(rt, level=l).cpu().numpy(), L.dims).astype(np.float64)
            ref = O.vcycle(lv, r, l)
            assert close(z, ref, dtype), (dims, l)


def solve_vs_oracle(dims, basis):
    lv = oracle_hierarchy(dims, 4, BETA)
    n = lv[0].n
    b = lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=0)
    x_o, info_o = O.gmres_ir(lv, b, tol=1e-12, restart=30)
    with hpg.Problem(*dims, beta=BETA, levels=4) as p:
        assert streamed(p.info[0])
        bt = torch.tensor(b, device=DEV)
        xt = torch.zeros_like(bt)
        info = hpg.gmres_ir_solve(p.h, bt, xt, tol=1e-12, restart=30, inner=hpg.HPG_FP32,
                                  basis=basis)
        x = xt.cpu().numpy()
    assert info["status"] == 0 and info["converged"] == 1
    assert np.linalg.norm(b - lv[0].A @ x) / np.linalg.norm(b) < 1e-12
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= 1e-8
    assert info["iterations"] <= 1.5 * info_o.iterations + 5


@pytest.mark.parametrize("basis", [hpg.HPG_FP32, hpg.HPG_BF16])
def test_streamed_mxp_solve_80cube_matches_oracle(basis):
    solve_vs_oracle((80, 80, 80), basis)


@pytest.mark.slow
def test_streamed_mxp_solve_128cube_matches_oracle():
    """The benchmark grid and solver settings, to 1e-12 against the oracle."""
    solve_vs_oracle((128, 128, 128), hpg.HPG_FP32)


@pytest.mark.parametrize("dims", GRIDS)
def test_halo_staged_phases_equal_plain_phases(dims):
    """HPG_OPT_GS_HALO: the streamed FP32 phases that stage z in shared memory
    give the plain phases' results bit for bit (smoother, V-cycle)."""
    with hpg.Problem(*dims, beta=BETA, levels=4) as p:
        for l in range(p.levels):
            info = p.info[l]
            r = random_vector(info["n"], seed=91 + l, dtype=np.float32)
            z0 = random_vector(info["n"], seed=92 + l, dtype=np.float32)
            rt = torch.tensor(to_storage(r, info["dims"]), device=DEV)
            out = []
            for opt in (0, 1):
                hpg.set_option(p.h, hpg.HPG_OPT_GS_HALO, opt)
                zt = torch.tensor(to_storage(z0, info["dims"]), device=DEV)
                hpg.mg_smooth(p.h, l, rt, zt, 2, False)
                out.append((zt, p.vcycle(rt, level=l)))
            hpg.set_option(p.h, hpg.HPG_OPT_GS_HALO, 0)
            torch.testing.assert_close(out[0][0], out[1][0], rtol=0, atol=0)
            torch.testing.assert_close(out[0][1], out[1][1], rtol=0, atol=0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_streamed_phases_with_misaligned_vectors(dtype):
    """The streamed phases move r and z as 16-byte vectors when both are
    16-byte aligned and row by row otherwise (caller pointers of the C ABI):
    r and z one element off a 16-byte boundary give the aligned results bit
    for bit (smoother from a given z, V-cycle); the aligned results are the
    ones checked against the oracle above."""
    dims = (82, 78, 84)
    with hpg.Problem(*dims, beta=BETA, levels=4) as p:
        info = p.info[0]
        assert streamed(info)
        ns = info["n_store"]
        r = random_vector(info["n"], seed=95, dtype=npdtype(dtype))
        z0 = random_vector(info["n"], seed=96, dtype=npdtype(dtype))
        rs = torch.tensor(to_storage(r, info["dims"]), device=DEV)
        zs = torch.tensor(to_storage(z0, info["dims"]), device=DEV)
        za = zs.clone()
        hpg.mg_smooth(p.h, 0, rs, za, 2, False)
        va = p.vcycle(rs, level=0)
        rb = torch.zeros(ns + 1, dtype=dtype, device=DEV)
        zb = torch.zeros(ns + 1, dtype=dtype, device=DEV)
        vb = torch.zeros(ns + 1, dtype=dtype, device=DEV)
        rb[1:] = rs
        zb[1:] = zs
        assert rb[1:].data_ptr() % 16 != 0 and zb[1:].data_ptr() % 16 != 0
        hpg.mg_smooth(p.h, 0, rb[1:], zb[1:], 2, False)
        hpg.mg_vcycle(p.h, 0, rb[1:], vb[1:])
        torch.testing.assert_close(zb[1:], za, rtol=0, atol=0)
        torch.testing.assert_close(vb[1:], va, rtol=0, atol=0)


def test_halo_staged_solve_equals_plain_solve():
    dims = (80, 80, 80)
    n = 80 ** 3
    b = torch.tensor(random_vector(n, seed=5), device=DEV)
    with hpg.Problem(*dims, beta=BETA) as p:
        xs, its = [], []
        for opt in (0, 1):
            hpg.set_option(p.h, hpg.HPG_OPT_GS_HALO, opt)
            x = torch.zeros_like(b)
            info = hpg.gmres_ir_solve(p.h, b, x, tol=1e-10, inner=hpg.HPG_FP32)
            assert info["status"] == 0
            xs.append(x)
            its.append(info["iterations"])
    assert its[0] == its[1]
    torch.testing.assert_close(xs[0], xs[1], rtol=0, atol=0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_streamed_vcycle_symmetric_theta_scaled(dtype):
    """beta = 0 (the paper's benchmarked symmetric matrix) with a per-cell
    diagonal scale theta ~ U(0.9, 1.1) at a streamed size: the V-cycle from
    every level against the oracle's (theta injected on the coarse levels)."""
    dims = (80, 80, 80)
    theta = np.random.default_rng(21).uniform(0.9, 1.1, 80 ** 3)
    lv = O.build_hierarchy(*dims, levels=4, beta=0.0, theta=theta)
    with hpg.Problem(*dims, beta=0.0, theta=theta) as p:
        assert streamed(p.info[0])
        for l, L in enumerate(lv):
            r = random_vector(L.n, seed=101 + l, dtype=npdtype(dtype)).astype(np.float64)
            rt = torch.tensor(to_storage(r, L.dims), dtype=dtype, device=DEV)
            z = to_natural(p.vcycle(rt, level=l).cpu().numpy(), L.dims).astype(np.float64)
            assert close(z, O.vcycle(lv, r, l), dtype), l


def test_streamed_fp64_gmres_matches_oracle():
    """Plain FP64 GMRES(30) (Algorithm 2) at a streamed size: its sweeps on the
    streamed level run as the pipelined kernel; x against the oracle's at 1e-8
    and the iteration counts within a few steps."""
    dims = (80, 80, 80)
    lv = oracle_hierarchy(dims, 4, BETA)
    n = lv[0].n
    b = lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=2)
    x_o, info_o = O.gmres_ir(lv, b, tol=1e-12, restart=30)
    with hpg.Problem(*dims, beta=BETA) as p:
        bt = torch.tensor(b, device=DEV)
        xt = torch.zeros_like(bt)
        info = hpg.gmres_ir_solve(p.h, bt, xt, tol=1e-12, restart=30, inner=hpg.HPG_FP64)
        x = xt.cpu().numpy()
    assert info["status"] == 0
    assert np.linalg.norm(b - lv[0].A @ x) / np.linalg.norm(b) < 1e-12
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= 1e-8
    assert abs(info["iterations"] - info_o.iterations) <= 3


@pytest.mark.parametrize("pre,post", [(0, 2), (2, 1), (1, 3)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_streamed_vcycle_sweep_counts(pre, post, dtype):
    """Other pre/post sweep counts at a streamed size: pre = 0 starts from a
    zeroed z with no first phase fused into the restriction; more sweeps
    repeat the full phases."""
    dims = (80, 80, 80)
    lv = oracle_hierarchy(dims, 4, BETA)
    with hpg.Problem(*dims, beta=BETA, levels=4, pre_sweeps=pre, post_sweeps=post) as p:
        r = random_vector(lv[0].n, seed=111, dtype=npdtype(dtype)).astype(np.float64)
        rt = torch.tensor(to_storage(r, lv[0].dims), dtype=dtype, device=DEV)
        z = to_natural(p.vcycle(rt).cpu().numpy(), lv[0].dims).astype(np.float64)
    assert close(z, O.vcycle(lv, r, 0, pre, post), dtype)


def test_streamed_mxp_solve_fp16_basis_matches_oracle():
    solve_vs_oracle((80, 80, 80), hpg.HPG_FP16)
