"""Many right-hand sides (hpg_*_batch) and many systems in one graph launch
(hpg_batch_*): stencil kernels bitwise equal to the single-vector ones in
every launch shape, batched GMRES-IR against the oracle per right-hand side,
the multi-system graph against per-system solves."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from oracle import hpg_oracle as O  # noqa: E402
from paper_2507_11512_gb300 import batch  # noqa: E402
from tests.gpu_helpers import oracle_hierarchy  # noqa: E402
from workloads import batch_systems, rhs_noise, x_true  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def shapes(R):
    lprs = sorted({1, min(2, R), R})
    return [(l, b) for l in lprs for b in (64, 256)]


def rvec(p, level, R, seed, padding_zero=True):
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = p.info[level]["n"]
    nat = torch.randn(R, n, generator=g, dtype=torch.float32).to(DEV)
    st = torch.empty(p.n_store(level), R, dtype=torch.float32, device=DEV)
    batch.permute_batch(p.h, level, 0, R, nat, st)
    return nat, st


@pytest.mark.parametrize("R", [1, 2, 4, 8])
def test_spmv_and_vcycle_columns_equal_single_vector_kernels(R):
    dims = (24, 20, 28)
    with hpg.Problem(*dims, beta=0.5) as p:
        for level in range(p.levels):
            _, X = rvec(p, level, R, 7 + level)
            for kind in (batch.KIND_SPMV, batch.KIND_GS):
                for lpr, blk in shapes(R):
                    batch.set_shape(p.h, level, kind, R, lpr, blk)
                    if kind == batch.KIND_SPMV:
                        Y = torch.empty_like(X)
                        batch.spmv_batch(p.h, level, X, Y)
                        ref = [p.spmv(X[:, r].contiguous(), level=level) for r in range(R)]
                    else:
                        Y = torch.empty_like(X)
                        batch.vcycle_batch(p.h, level, X, Y)
                        ref = [p.vcycle(X[:, r].contiguous(), level=level) for r in range(R)]
                    for r in range(R):
                        assert torch.equal(Y[:, r], ref[r]), (level, kind, lpr, blk, r)
                batch.set_shape(p.h, level, kind, R, 0, 0)


def test_permute_batch_round_trip():
    with hpg.Problem(12, 10, 14) as p:
        nat, st = rvec(p, 0, 4, 3)
        back = torch.empty_like(nat)
        batch.permute_batch(p.h, 0, 1, 4, st, back)
        assert torch.equal(back, nat)
        for r in range(4):
            assert torch.equal(st[:, r], p.to_storage(nat[r].contiguous()))


@pytest.mark.parametrize("dims,beta", [((16, 16, 16), 0.5), ((24, 20, 28), 0.0)])
def test_batched_solve_matches_oracle_per_rhs(dims, beta):
    lv = oracle_hierarchy(dims, 4, beta)
    n = lv[0].n
    R = 8
    rhs = [lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=r) for r in range(R - 2)]
    rhs.append(np.zeros(n))                                    # b = 0: x = 0 at once
    rhs.append(1e-6 * (lv[0].A @ x_true(n)))                   # another scale
    B = torch.tensor(np.stack(rhs), device=DEV)
    X = torch.zeros_like(B)
    with hpg.Problem(*dims, beta=beta) as p:
        infos = batch.solve_batch(p.h, B, X, tol=1e-12)
    x = X.cpu().numpy()
    for r in range(R):
        assert infos[r]["converged"] == 1 and infos[r]["status"] == 0, (r, infos[r])
        if r == R - 2:
            assert np.all(x[r] == 0.0) and infos[r]["iterations"] == 0
            continue
        res = np.linalg.norm(rhs[r] - lv[0].A @ x[r]) / np.linalg.norm(rhs[r])
        assert res < 1e-12
        x_o, _ = O.gmres_ir(lv, rhs[r], tol=1e-12, restart=30)
        assert np.linalg.norm(x[r] - x_o) / np.linalg.norm(x_o) <= 1e-8


def test_batched_solve_graph_equals_eager_and_is_deterministic():
    dims = (16, 16, 16)
    lv = oracle_hierarchy(dims, 4, 0.5)
    n = lv[0].n
    B = torch.tensor(np.stack([lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=r)
                               for r in range(4)]), device=DEV)
    with hpg.Problem(*dims, beta=0.5) as p:
        Xg = torch.zeros_like(B)
        ig = batch.solve_batch(p.h, B, Xg, tol=1e-10)
        Xg2 = torch.zeros_like(B)
        batch.solve_batch(p.h, B, Xg2, tol=1e-10)
        hpg.set_execution(p.h, hpg.HPG_EXEC_EAGER)
        Xe = torch.zeros_like(B)
        ie = batch.solve_batch(p.h, B, Xe, tol=1e-10)
    assert torch.equal(Xg, Xe) and torch.equal(Xg, Xg2)
    assert [i["iterations"] for i in ig] == [i["iterations"] for i in ie]
    assert ig[0]["graph_launches"] == 1 and ie[0]["graph_launches"] == 0
    assert ig[0]["kernel_launches"] == ie[0]["kernel_launches"]


def test_batch_of_systems_in_one_graph_equals_per_system_solves():
    spec = batch_systems(4, 4, seed=1)
    for s in spec:   # small grids for the test
        e = {24: 12, 32: 16, 48: 8, 64: 16, 96: 24}[s["dims"][0]]
        s["dims"] = (e, e, e)
        s["rhs"] = np.random.default_rng(5).standard_normal((4, e ** 3))
    probs = [hpg.Problem(*s["dims"], beta=s["beta"]) for s in spec]
    try:
        Bs = [torch.tensor(s["rhs"], device=DEV) for s in spec]
        ref = []
        for p, b in zip(probs, Bs):
            x = torch.zeros_like(b)
            info = batch.solve_batch(p.h, b, x, tol=1e-9)
            ref.append((x, info))
        with batch.BatchSolver(probs, 4, tune_shapes=True) as bsol:
            Xs = [torch.zeros_like(b) for b in Bs]
            bsol.tune(Bs, Xs, tol=1e-9)
            Xs = [torch.zeros_like(b) for b in Bs]
            infos = bsol.solve(Bs, Xs, tol=1e-9)
            # tuned shapes give the same values as the default ones
            for (x_ref, i_ref), x, inf in zip(ref, Xs, infos):
                assert torch.equal(x, x_ref)
                assert [i["iterations"] for i in inf] == [i["iterations"] for i in i_ref]
                assert all(i["converged"] for i in inf)
            # a second call reuses the graph
            Xs2 = [torch.zeros_like(b) for b in Bs]
            bsol.solve(Bs, Xs2, tol=1e-9)
            assert all(torch.equal(a, b) for a, b in zip(Xs, Xs2))
            # while the batch owns the buffers, other shapes of batch solves are refused
            with pytest.raises(hpg.HpgError):
                batch.solve_batch(probs[0].h, Bs[0][:2].contiguous(),
                                  torch.zeros_like(Bs[0][:2]).contiguous(), tol=1e-9)
        for p in probs:
            for level in range(p.levels):
                lpr, blk = batch.get_shape(p.h, level, batch.KIND_GS, 4)
                assert lpr in (1, 2, 4) and blk in (64, 128, 256)
    finally:
        for p in probs:
            p.close()


def test_batch_invalid_arguments():
    with hpg.Problem(8, 8, 8) as p:
        B = torch.ones(3, 512, dtype=torch.float64, device=DEV)
        with pytest.raises(hpg.HpgError):
            batch.solve_batch(p.h, B, torch.zeros_like(B))   # nrhs 3
        with pytest.raises(hpg.HpgError):
            batch.set_shape(p.h, 0, 0, 4, 3, 64)
        with pytest.raises(hpg.HpgError):
            batch.set_shape(p.h, 0, 0, 4, 1, 100)
        with pytest.raises(hpg.HpgError):
            batch.BatchSolver([p, p], 4, tune_shapes=False)


def test_problem_outlives_its_batch():
    """A batch's graph points at its problems' buffers: while it exists the
    library refuses to destroy, rebuild or re-option those problems; after
    hpg_batch_destroy the same calls succeed and batched solves still work."""
    lib = hpg.load()
    pa, pb = hpg.Problem(16, 16, 16, beta=0.5), hpg.Problem(8, 8, 8, beta=0.25)
    try:
        solver = batch.BatchSolver([pa, pb], 2, restart=10)
        Bs = [torch.ones(2, 16 ** 3, dtype=torch.float64, device=DEV),
              torch.ones(2, 8 ** 3, dtype=torch.float64, device=DEV)]
        Xs = [torch.zeros_like(b) for b in Bs]
        ref = solver.solve(Bs, Xs, tol=1e-8)
        assert lib.hpg_destroy(pa.h) == hpg.HPG_ERR_STATE
        assert b"hpg_batch_destroy" in lib.hpg_last_error()
        assert lib.hpg_build_mg_hierarchy(pb.h, 4, 1, 1) == hpg.HPG_ERR_STATE
        assert lib.hpg_set_option(pa.h, hpg.HPG_OPT_PDL, 0) == hpg.HPG_ERR_STATE
        # the refused calls changed nothing: the batch solves as before
        for x in Xs:
            x.zero_()
        again = solver.solve(Bs, Xs, tol=1e-8)
        assert [[i["iterations"] for i in s] for s in again] == \
            [[i["iterations"] for i in s] for s in ref]
        solver.close()
        hpg.set_option(pa.h, hpg.HPG_OPT_PDL, 0)
        hpg.build_mg_hierarchy(pb.h, 4, 1, 1)
        x = torch.zeros_like(Bs[1])
        infos = batch.solve_batch(pb.h, Bs[1], x, tol=1e-8, restart=10)
        assert all(i["converged"] for i in infos)
    finally:
        pa.close()
        pb.close()


@pytest.mark.parametrize("pdl_rows", [16384, 1 << 30])
@pytest.mark.parametrize("R", [2, 8])
def test_streamed_size_system_columns_equal_single_vector_kernels(R, pdl_rows):
    """A 96^3 system (the batched workload's largest edge): its level-0 matrix
    streams from memory, level 1 is cached, levels 2-3 are read evict-last;
    every launch shape's columns equal the single-vector kernels bitwise.
    pdl_rows = 2^30 launches every phase programmatically, so each phase's
    matrix loads overlap the previous kernel and its gathers follow the
    grid-dependency wait directly: read through the non-coherent path, the
    level-0 columns of that configuration differed on GB300."""
    dims = (96, 96, 96)
    with hpg.Problem(*dims, beta=0.6) as p:
        assert p.n_store(0) * 27 * 8 > (96 << 20)
        hpg.set_option(p.h, hpg.HPG_OPT_PDL_ROWS, pdl_rows)
        for level in (0, 1):
            _, X = rvec(p, level, R, 30 + level)
            ref_s = [p.spmv(X[:, r].contiguous(), level=level) for r in range(R)]
            ref_v = [p.vcycle(X[:, r].contiguous(), level=level) for r in range(R)]
            for lpr, blk in shapes(R):
                for kind in (batch.KIND_SPMV, batch.KIND_GS):
                    batch.set_shape(p.h, level, kind, R, lpr, blk)
                Y = torch.empty_like(X)
                batch.spmv_batch(p.h, level, X, Y)
                Z = torch.empty_like(X)
                batch.vcycle_batch(p.h, level, X, Z)
                for r in range(R):
                    assert torch.equal(Y[:, r], ref_s[r]), (level, lpr, blk, r)
                    assert torch.equal(Z[:, r], ref_v[r]), (level, lpr, blk, r)
            for kind in (batch.KIND_SPMV, batch.KIND_GS):
                batch.set_shape(p.h, level, kind, R, 0, 0)


def test_batched_solve_same_with_every_phase_programmatic():
    dims = (96, 96, 96)
    g = torch.Generator(device="cpu").manual_seed(11)
    n = dims[0] * dims[1] * dims[2]
    B = torch.randn(2, n, generator=g, dtype=torch.float64).to(DEV)
    with hpg.Problem(*dims, beta=0.6) as p:
        xs, its = [], []
        for rows in (16384, 1 << 30):
            hpg.set_option(p.h, hpg.HPG_OPT_PDL_ROWS, rows)
            X = torch.zeros_like(B)
            infos = batch.solve_batch(p.h, B, X, tol=1e-8)
            assert all(i["converged"] for i in infos)
            xs.append(X)
            its.append([i["iterations"] for i in infos])
    assert its[0] == its[1]
    assert torch.equal(xs[0], xs[1])


def test_streamed_size_batched_solve_matches_oracle():
    dims, beta = (96, 96, 96), 0.6
    lv = oracle_hierarchy(dims, 4, beta)
    n = lv[0].n
    rhs = [lv[0].A @ x_true(n) + rhs_noise(n, 1e-3, seed=3), rhs_noise(n, 1.0, seed=4)]
    B = torch.tensor(np.stack(rhs), device=DEV)
    X = torch.zeros_like(B)
    with hpg.Problem(*dims, beta=beta) as p:
        infos = batch.solve_batch(p.h, B, X, tol=1e-12)
    x = X.cpu().numpy()
    for r in range(2):
        assert infos[r]["converged"] == 1 and infos[r]["status"] == 0, (r, infos[r])
        assert np.linalg.norm(rhs[r] - lv[0].A @ x[r]) / np.linalg.norm(rhs[r]) < 1e-12
        x_o, _ = O.gmres_ir(lv, rhs[r], tol=1e-12, restart=30)
        assert np.linalg.norm(x[r] - x_o) / np.linalg.norm(x_o) <= 1e-8
