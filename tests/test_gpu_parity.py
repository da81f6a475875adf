"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from oracle import hpg_oracle as O  # noqa: E402
from tests.gpu_helpers import (FP32_ELEM, FP32_REL, FP64_REL, abs_matvec,  # noqa: E402
                               oracle_hierarchy, storage_layout, to_natural, to_storage)
from workloads import random_vector, rhs_noise, x_true  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
# grids that span several 256-row blocks and leave ragged colour blocks;
# odd edges stop the coarsening early
GRIDS = [(16, 16, 16), (24, 20, 28), (12, 12, 12), (33, 17, 9), (1, 1, 1), (2, 2, 2),
         (40, 36, 28)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def gpu(v, dtype):
    return torch.tensor(v, dtype=dtype, device=DEV)


@pytest.mark.parametrize("dims", GRIDS)
def test_layout_and_permute(dims):
    with hpg.Problem(*dims, beta=0.5) as p:
        idx, ns, offs = storage_layout(dims)
        info = p.info[0]
        assert info["n_store"] == ns
        assert info["colour_offset"] == offs
        assert info["nnz"] == O.build_matrix(*dims).nnz
        n = idx.size
        v = np.arange(n, dtype=np.float64) + 1.0
        st = p.to_storage(gpu(v, torch.float64)).cpu().numpy()
        np.testing.assert_array_equal(st, to_storage(v, dims))
        back = p.to_natural(gpu(st, torch.float64)).cpu().numpy()
        np.testing.assert_array_equal(back, v)
        st32 = p.to_storage(gpu(v, torch.float64), dtype=torch.float32).cpu().numpy()
        np.testing.assert_array_equal(st32, to_storage(v.astype(np.float32), dims))


@pytest.mark.parametrize("dims", GRIDS)
@pytest.mark.parametrize("beta", [0.0, 0.5, -1.0])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spmv_parity_all_levels(dims, beta, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    lv = oracle_hierarchy(dims, 4, beta)
    with hpg.Problem(*dims, beta=beta, levels=4) as p:
        assert p.levels == len(lv)
        for l, L in enumerate(lv):
            x = random_vector(L.n, seed=11 + l, dtype=np.float64 if prec == "fp64"
                              else np.float32).astype(np.float64)
            y = p.spmv(gpu(to_storage(x, L.dims), dt), level=l).cpu().numpy()
            y = to_natural(y, L.dims).astype(np.float64)
            ref = L.A @ x
            scale = abs_matvec(L.A, x)
            err = np.abs(y - ref)
            if prec == "fp64":
                assert np.all(err <= FP64_REL * scale + 1e-300)
            else:
                assert np.all(err <= FP32_ELEM * scale)
                assert np.linalg.norm(y - ref) <= FP32_REL * np.linalg.norm(ref) + 1e-30


@pytest.mark.parametrize("dims", [(16, 16, 16), (24, 20, 28), (12, 12, 12), (8, 8, 8),
                                  (40, 36, 28), (33, 17, 9)])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_vcycle_parity_fp64(dims, beta):
    lv = oracle_hierarchy(dims, 4, beta)
    with hpg.Problem(*dims, beta=beta, levels=4) as p:
        for l, L in enumerate(lv):
            r = random_vector(L.n, seed=21 + l)
            z = p.vcycle(gpu(to_storage(r, L.dims), torch.float64), level=l).cpu().numpy()
            z = to_natural(z, L.dims)
            ref = O.vcycle(lv, r, l)
            assert np.abs(z - ref).max() <= FP64_REL * np.abs(ref).max()


@pytest.mark.parametrize("dims", [(16, 16, 16), (24, 20, 28), (40, 36, 28)])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_vcycle_parity_fp32(dims, beta):
    lv = oracle_hierarchy(dims, 4, beta)
    with hpg.Problem(*dims, beta=beta, levels=4) as p:
        for l, L in enumerate(lv):
            r = random_vector(L.n, seed=31 + l, dtype=np.float32).astype(np.float64)
            z = p.vcycle(gpu(to_storage(r, L.dims), torch.float32), level=l).cpu().numpy()
            z = to_natural(z, L.dims).astype(np.float64)
            ref = O.vcycle(lv, r, l)
            assert np.linalg.norm(z - ref) <= FP32_REL * np.linalg.norm(ref)


def test_vcycle_pre_post_sweeps():
    dims = (16, 16, 16)
    for pre, post in [(2, 1), (0, 2), (1, 0), (3, 3)]:
        lv = O.build_hierarchy(*dims, 4, 0.5)
        with hpg.Problem(*dims, beta=0.5, levels=4, pre_sweeps=pre, post_sweeps=post) as p:
            r = random_vector(lv[0].n, seed=5)
            z = to_natural(p.vcycle(gpu(to_storage(r, dims), torch.float64)).cpu().numpy(),
                           dims)
            ref = O.vcycle(lv, r, 0, pre, post)
            assert np.abs(z - ref).max() <= FP64_REL * np.abs(ref).max()


def solve_gpu(dims, beta, b, inner, tol=1e-9, restart=30, maxit=10000, x0=None, levels=4):
    with hpg.Problem(*dims, beta=beta, levels=levels) as p:
        bt = gpu(b, torch.float64)
        xt = torch.zeros_like(bt) if x0 is None else gpu(x0, torch.float64)
        info = hpg.gmres_ir_solve(p.h, bt, xt, tol=tol, restart=restart, maxit=maxit,
                                  inner=inner)
        return xt.cpu().numpy(), info


def test_fp64_gmres_16cube_matches_oracle():
    # plain FP64 GMRES(30), 4 levels, b = A * 1, x0 = 0, tol 1e-9
    dims, beta = (16, 16, 16), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    b = lv[0].A @ x_true(lv[0].n)
    x_o, info_o = O.gmres_ir(lv, b, tol=1e-9, restart=30)
    x, info = solve_gpu(dims, beta, b, hpg.HPG_FP64)
    assert info["status"] == 0 and info["converged"] == 1
    assert info["rel_residual"] < 1e-9
    assert abs(info["iterations"] - info_o.iterations) <= 1
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= 1e-8
    assert np.abs(x - 1.0).max() < 1e-6


@pytest.mark.parametrize("dims,beta", [((16, 16, 16), 0.5), ((24, 20, 28), 0.0),
                                       ((32, 32, 32), 0.5)])
def test_mxp_gmres_ir_matches_oracle(dims, beta):
    lv = oracle_hierarchy(dims, 4, beta)
    n = lv[0].n
    b = lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=0)
    x_o, info_o = O.gmres_ir(lv, b, tol=1e-12, restart=30)
    x, info = solve_gpu(dims, beta, b, hpg.HPG_FP32, tol=1e-12)
    assert info["status"] == 0
    r = np.linalg.norm(b - lv[0].A @ x) / np.linalg.norm(b)
    assert r < 1e-12
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= 1e-8
    # the mixed-precision solve converges at a comparable rate (Sec. 4: n_d/n_ir ~ 0.97)
    assert info["iterations"] <= 1.5 * info_o.iterations + 5


@pytest.mark.parametrize("inner", [hpg.HPG_FP64, hpg.HPG_FP32])
def test_solve_tolerance_1e9_true_residual(inner):
    dims, beta = (24, 24, 24), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    n = lv[0].n
    b = lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=0)
    x, info = solve_gpu(dims, beta, b, inner)
    r = np.linalg.norm(b - lv[0].A @ x) / np.linalg.norm(b)
    assert info["converged"] == 1 and r < 1e-9
    assert abs(r - info["rel_residual"]) <= 1e-3 * r


def test_solve_zero_rhs():
    x, info = solve_gpu((8, 8, 8), 0.5, np.zeros(512), hpg.HPG_FP32, x0=np.ones(512))
    assert info["status"] == 0 and info["iterations"] == 0
    assert np.all(x == 0.0)


def test_solve_single_point():
    x, info = solve_gpu((1, 1, 1), 0.0, np.array([3.0]), hpg.HPG_FP64, tol=1e-12)
    assert info["status"] == 0 and info["iterations"] == 1
    assert x[0] == pytest.approx(3.0 / 26.0, rel=1e-15)


def test_solve_maxit_not_converged():
    dims = (16, 16, 16)
    b = random_vector(4096, seed=3)
    x, info = solve_gpu(dims, 0.5, b, hpg.HPG_FP32, tol=1e-12, restart=5, maxit=7)
    assert info["status"] == hpg.HPG_ERR_NOT_CONVERGED
    assert info["iterations"] == 7 and info["converged"] == 0
    lv = oracle_hierarchy(dims, 4, 0.5)
    x_o, info_o = O.gmres_ir(lv, b, tol=1e-12, restart=5, maxit=7)
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) < 1e-4


def test_warm_start_at_solution():
    dims = (8, 8, 8)
    lv = oracle_hierarchy(dims, 4, 0.5)
    xs = random_vector(512, seed=9)
    x, info = solve_gpu(dims, 0.5, lv[0].A @ xs, hpg.HPG_FP64, x0=xs)
    assert info["status"] == 0 and info["iterations"] == 0


def test_host_buffers_match_device():
    dims, beta = (16, 12, 8), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    b = lv[0].A @ x_true(lv[0].n) + rhs_noise(lv[0].n, 1e-3)
    x_dev, info_d = solve_gpu(dims, beta, b, hpg.HPG_FP32)
    with hpg.Problem(*dims, beta=beta) as p:
        bh = torch.tensor(b).pin_memory()
        xh = torch.zeros_like(bh).pin_memory()
        info_h = hpg.gmres_ir_solve(p.h, bh, xh, inner=hpg.HPG_FP32)
        xn = np.zeros_like(b)
        info_n = hpg.gmres_ir_solve(p.h, b, xn, inner=hpg.HPG_FP32)
    np.testing.assert_array_equal(xh.numpy(), x_dev)
    np.testing.assert_array_equal(xn, x_dev)
    assert info_h["iterations"] == info_d["iterations"] == info_n["iterations"]


def test_deterministic_bitwise():
    dims = (24, 20, 28)
    b = random_vector(24 * 20 * 28, seed=4)
    x1, i1 = solve_gpu(dims, 0.5, b, hpg.HPG_FP32)
    x2, i2 = solve_gpu(dims, 0.5, b, hpg.HPG_FP32)
    np.testing.assert_array_equal(x1, x2)
    assert i1["iterations"] == i2["iterations"]


def test_invalid_arguments():
    with hpg.Problem(8, 8, 8) as p:
        b = torch.ones(512, dtype=torch.float64, device=DEV)
        x = torch.zeros_like(b)
        for kw in [dict(tol=0.0), dict(restart=0), dict(restart=65), dict(maxit=-1),
                   dict(inner=hpg.HPG_FP32, basis=hpg.HPG_FP64)]:
            with pytest.raises(hpg.HpgError):
                hpg.gmres_ir_solve(p.h, b, x, **kw)
        with pytest.raises(hpg.HpgError):
            hpg.spmv(p.h, 9, b, x)
        with pytest.raises(hpg.HpgError):
            hpg.mg_vcycle(p.h, 0, b, b)
    for dims in [(0, 4, 4), (4, -1, 4)]:
        with pytest.raises(hpg.HpgError):
            hpg.setup_problem(*dims)
    with pytest.raises(hpg.HpgError):
        hpg.setup_problem(4, 4, 4, beta=1.5)
    with pytest.raises(hpg.HpgError):
        hpg.setup_problem(2000, 2000, 2000)


def test_theta_scaled_diagonal():
    dims = (12, 12, 12)
    rng = np.random.default_rng(0)
    theta = rng.uniform(0.9, 1.1, 12 ** 3)
    lv = O.build_hierarchy(*dims, 4, 0.25, theta)
    with hpg.Problem(*dims, beta=0.25, theta=theta) as p:
        for l, L in enumerate(lv):
            r = random_vector(L.n, seed=l)
            z = to_natural(p.vcycle(gpu(to_storage(r, L.dims), torch.float64), l).cpu().numpy(),
                           L.dims)
            ref = O.vcycle(lv, r, l)
            assert np.abs(z - ref).max() <= FP64_REL * np.abs(ref).max()


@pytest.mark.parametrize("inner", [hpg.HPG_FP32, hpg.HPG_FP64])
def test_graph_and_eager_paths_agree(inner):
    # the whole-solve CUDA graph (conditional WHILE/IF nodes, programmatic
    # launches) and the host-driven path run the same deterministic kernels
    dims, beta = (24, 20, 28), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    n = lv[0].n
    b = lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=0)
    with hpg.Problem(*dims, beta=beta) as p:
        bt = gpu(b, torch.float64)
        xg = torch.zeros_like(bt)
        ig = hpg.gmres_ir_solve(p.h, bt, xg, tol=1e-10, restart=12, inner=inner)
        hpg.set_execution(p.h, hpg.HPG_EXEC_EAGER)
        xq = torch.zeros_like(bt)
        iq = hpg.gmres_ir_solve(p.h, bt, xq, tol=1e-10, restart=12, inner=inner)
        hpg.set_execution(p.h, hpg.HPG_EXEC_GRAPH)
        hpg.set_profiling(p.h, True)
        xe = torch.zeros_like(bt)
        ie = hpg.gmres_ir_solve(p.h, bt, xe, tol=1e-10, restart=12, inner=inner)
        rep = hpg.profile_report(p.h)
        hpg.set_profiling(p.h, False)
    assert ig["graph_launches"] == 1 and ie["graph_launches"] == 0
    assert ig["iterations"] == ie["iterations"] and ig["restarts"] == ie["restarts"]
    assert ig["kernel_launches"] == ie["kernel_launches"]
    torch.testing.assert_close(xg, xe, rtol=0, atol=0)
    torch.testing.assert_close(xg, xq, rtol=0, atol=0)
    assert iq["graph_launches"] == 0 and iq["kernel_launches"] == ig["kernel_launches"]
    names = {r["name"] for r in rep}
    assert {"gs_colour_phase", "restrict", "prolong", "spmv", "cgs2_gemvt", "cgs2_reorth",
            "cgs2_final_givens", "arnoldi_scale", "residual_fp64"} <= names
    # with the coarse-level cluster kernel the whole (small) V-cycle is one kernel
    with hpg.Problem(*dims, beta=beta) as p:
        hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CLUSTER, 1)
        hpg.set_profiling(p.h, True)
        xc = torch.zeros_like(bt)
        ic = hpg.gmres_ir_solve(p.h, bt, xc, tol=1e-10, restart=12, inner=inner)
        repc = hpg.profile_report(p.h)
    torch.testing.assert_close(xg, xc, rtol=0, atol=0)
    vc = [r for r in repc if r["name"] == "vcycle_coarse_cluster"][0]
    assert vc["launches"] == ic["iterations"] + ic["restarts"]
    with hpg.Problem(*dims, beta=beta) as p:
        hpg.set_profiling(p.h, True)
        xp = torch.zeros_like(bt)
        ip = hpg.gmres_ir_solve(p.h, bt, xp, tol=1e-10, restart=12, inner=inner)
        rep = hpg.profile_report(p.h)
    torch.testing.assert_close(xg, xp, rtol=0, atol=0)
    names = {r["name"] for r in rep}
    assert {"gs_colour_phase", "restrict", "prolong"} <= names
    gs0 = [r for r in rep if r["name"] == "gs_colour_phase" and r["level"] == 0][0]
    # 30 level-0 phases per V-cycle (15 per symmetric sweep); in the inner
    # steps the first one (colour 0 from zero) comes with the kernel that
    # writes the V-cycle's input, the cycle-end V-cycle launches all 30
    assert gs0["launches"] == ip["iterations"] * 29 + ip["restarts"] * 30
    assert gs0["total_ms"] > 0 and gs0["bytes"] > 0


def test_repeated_solves_recapture():
    dims = (16, 16, 16)
    lv = oracle_hierarchy(dims, 4, 0.5)
    b = lv[0].A @ x_true(lv[0].n)
    with hpg.Problem(*dims, beta=0.5) as p:
        bt = gpu(b, torch.float64)
        res = []
        for restart, inner in [(30, hpg.HPG_FP32), (10, hpg.HPG_FP32), (30, hpg.HPG_FP64),
                               (30, hpg.HPG_FP32), (30, hpg.HPG_FP32)]:
            x = torch.zeros_like(bt)
            info = hpg.gmres_ir_solve(p.h, bt, x, restart=restart, inner=inner)
            assert info["status"] == 0 and info["rel_residual"] < 1e-9
            res.append(x.cpu().numpy())
        np.testing.assert_array_equal(res[0], res[3])
        np.testing.assert_array_equal(res[3], res[4])


@pytest.mark.parametrize("dims", [(16, 16, 16), (24, 20, 28), (40, 36, 28), (64, 64, 64),
                                  (33, 17, 9)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_cluster_vcycle_equals_phase_launches(dims, dtype):
    # coarse levels in one cluster kernel vs one launch per phase: same
    # phases, same arithmetic, so the results are equal
    with hpg.Problem(*dims, beta=0.5) as p:
        for l in range(p.levels):
            info = p.info[l]
            r = random_vector(info["n"], seed=7 + l,
                              dtype=np.float64 if dtype == torch.float64 else np.float32)
            rt = torch.tensor(to_storage(r, info["dims"]), dtype=dtype, device=DEV)
            hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CLUSTER, 1)
            z1 = p.vcycle(rt, l)
            hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CLUSTER, 0)
            z2 = p.vcycle(rt, l)
            np.testing.assert_array_equal(z1.cpu().numpy(), z2.cpu().numpy())


def test_cluster_vcycle_sweep_variants():
    dims = (32, 32, 32)
    for pre, post in [(0, 1), (2, 2), (1, 3)]:
        with hpg.Problem(*dims, beta=0.5, pre_sweeps=pre, post_sweeps=post) as p:
            r = torch.tensor(to_storage(random_vector(32 ** 3, seed=2), dims), device=DEV)
            hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CLUSTER, 1)
            z1 = p.vcycle(r)
            hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CLUSTER, 0)
            z2 = p.vcycle(r)
            np.testing.assert_array_equal(z1.cpu().numpy(), z2.cpu().numpy())


@pytest.mark.parametrize("inner", [hpg.HPG_FP32, hpg.HPG_FP64])
def test_solve_same_with_and_without_cluster_vcycle(inner):
    dims, beta = (48, 40, 32), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    b = lv[0].A @ x_true(lv[0].n) + rhs_noise(lv[0].n, 1e-3)
    with hpg.Problem(*dims, beta=beta) as p:
        bt = gpu(b, torch.float64)
        hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CLUSTER, 1)
        x1 = torch.zeros_like(bt)
        i1 = hpg.gmres_ir_solve(p.h, bt, x1, inner=inner)
        hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CLUSTER, 0)
        x2 = torch.zeros_like(bt)
        i2 = hpg.gmres_ir_solve(p.h, bt, x2, inner=inner)
        hpg.set_option(p.h, hpg.HPG_OPT_PDL, 0)
        x3 = torch.zeros_like(bt)
        i3 = hpg.gmres_ir_solve(p.h, bt, x3, inner=inner)
    assert i1["iterations"] == i2["iterations"] == i3["iterations"]
    np.testing.assert_array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    np.testing.assert_array_equal(x2.cpu().numpy(), x3.cpu().numpy())
    r = np.linalg.norm(b - lv[0].A @ x1.cpu().numpy()) / np.linalg.norm(b)
    assert r < 1e-9


@pytest.mark.parametrize("dims", [(16, 16, 16), (24, 20, 28), (40, 36, 28), (64, 64, 64),
                                  (96, 96, 96), (128, 128, 128), (12, 12, 12), (2, 2, 2)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_coarsest_sweep_in_one_cta_equals_phase_launches(dims, dtype):
    # HPG_OPT_COARSE_CTA: the coarsest level's sweep in one CTA (z in shared
    # memory) against one launch per colour phase: same phases, same order;
    # HPG_OPT_PDL_ROWS: programmatic launches of larger phases change nothing
    with hpg.Problem(*dims, beta=0.5) as p:
        for l in range(p.levels):
            info = p.info[l]
            r = random_vector(info["n"], seed=17 + l,
                              dtype=np.float64 if dtype == torch.float64 else np.float32)
            rt = torch.tensor(to_storage(r, info["dims"]), dtype=dtype, device=DEV)
            hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CTA, 1)
            z1 = p.vcycle(rt, l)
            hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CTA, 0)
            z2 = p.vcycle(rt, l)
            torch.testing.assert_close(z1, z2, rtol=0, atol=0)
            hpg.set_option(p.h, hpg.HPG_OPT_PDL_ROWS, 1 << 30)
            z3 = p.vcycle(rt, l)
            hpg.set_option(p.h, hpg.HPG_OPT_PDL_ROWS, 16384)
            torch.testing.assert_close(z1, z3, rtol=0, atol=0)


@pytest.mark.parametrize("inner", [hpg.HPG_FP32, hpg.HPG_FP64])
def test_solve_same_with_and_without_coarsest_cta(inner):
    dims, beta = (64, 64, 64), 0.5
    lv = oracle_hierarchy(dims, 4, beta)
    b = lv[0].A @ x_true(lv[0].n) + rhs_noise(lv[0].n, 1e-3)
    with hpg.Problem(*dims, beta=beta) as p:
        bt = gpu(b, torch.float64)
        xs = []
        for opt in (1, 0):
            hpg.set_option(p.h, hpg.HPG_OPT_COARSE_CTA, opt)
            hpg.set_option(p.h, hpg.HPG_OPT_PDL_ROWS, (1 << 30) if opt else 16384)
            x = torch.zeros_like(bt)
            info = hpg.gmres_ir_solve(p.h, bt, x, inner=inner)
            assert info["status"] == 0
            xs.append(x)
    torch.testing.assert_close(xs[0], xs[1], rtol=0, atol=0)
