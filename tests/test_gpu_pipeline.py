"""Pipelined symmetric sweep (HPG_OPT_GS_PIPELINE) on levels whose matrix
streams from memory: bitwise equal to the phase-by-phase sweep in the
smoother, the V-cycle and whole solves, over repeated launches."""

import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
GS_PIPELINE = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def storage_vec(p, dtype, seed, level=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    nat = torch.randn(p.info[level]["n"], generator=g, dtype=torch.float64).to(DEV)
    return p.to_storage(nat, level=level, dtype=dtype)


@pytest.mark.parametrize("dims", [(80, 80, 80), (82, 78, 84)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_pipelined_smoother_equals_phase_launches(dims, dtype):
    with hpg.Problem(*dims, beta=0.5, levels=3) as p:
        r = storage_vec(p, dtype, 1)
        z0 = storage_vec(p, dtype, 2)
        out = {}
        for pipe in (0, 2):
            hpg.set_option(p.h, GS_PIPELINE, pipe)
            for sweeps, zero in [(1, True), (2, False), (1, False)]:
                z = z0.clone()
                hpg.mg_smooth(p.h, 0, r, z, sweeps, zero)
                out[(pipe, sweeps, zero)] = z
            # repeated launches (the sweep kernel's epochs) give the same values
            z = z0.clone()
            for _ in range(3):
                hpg.mg_smooth(p.h, 0, r, z, 1, False)
            out[(pipe, "x3")] = z
        for key in [(1, True), (2, False), (1, False), ("x3",)]:
            a = out[(0,) + key] if key != ("x3",) else out[(0, "x3")]
            b = out[(2,) + key] if key != ("x3",) else out[(2, "x3")]
            assert torch.equal(a, b), key
        assert torch.isfinite(out[(2, "x3")]).all()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_pipelined_vcycle_equals_phase_launches(dtype):
    with hpg.Problem(80, 80, 80, beta=0.5) as p:
        r = storage_vec(p, dtype, 3)
        zs = []
        for pipe in (0, 2, 3):
            hpg.set_option(p.h, GS_PIPELINE, pipe)
            zs.append(p.vcycle(r))
        assert torch.equal(zs[0], zs[1]) and torch.equal(zs[0], zs[2])


@pytest.mark.parametrize("inner", [hpg.HPG_FP32, hpg.HPG_FP64])
def test_pipelined_solve_equals_phase_launches(inner):
    dims = (80, 80, 80)
    n = 80 ** 3
    with hpg.Problem(*dims, beta=0.5) as p:
        ones = torch.ones(n, dtype=torch.float64, device=DEV)
        b = p.to_natural(p.spmv(p.to_storage(ones)))
        res = []
        for pipe in (0, 2, 3):
            hpg.set_option(p.h, GS_PIPELINE, pipe)
            x = torch.zeros_like(b)
            info = hpg.gmres_ir_solve(p.h, b, x, tol=1e-9, inner=inner)
            assert info["status"] == 0 and info["converged"] == 1
            res.append((x, info["iterations"]))
        assert torch.equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]
        assert torch.equal(res[0][0], res[2][0]) and res[0][1] == res[2][1]


@pytest.mark.parametrize("dims", [(16, 16, 16), (33, 17, 9), (2, 2, 2), (24, 20, 28)])
def test_pipelined_sweeps_on_every_level_small_grids(dims):
    with hpg.Problem(*dims, beta=0.5) as p:
        for level in range(p.levels):
            r = storage_vec(p, torch.float32, 5 + level, level)
            zs = []
            for pipe in (0, 3):
                hpg.set_option(p.h, GS_PIPELINE, pipe)
                zs.append(p.vcycle(r, level=level))
                z = torch.zeros_like(r)
                hpg.mg_smooth(p.h, level, r, z, 2, True)
                zs.append(z)
            assert torch.equal(zs[0], zs[2]) and torch.equal(zs[1], zs[3])


def test_pipeline_option_values():
    with hpg.Problem(8, 8, 8) as p:
        for v in (0, 1, 2):
            hpg.set_option(p.h, GS_PIPELINE, v)
        with pytest.raises(hpg.HpgError):
            hpg.set_option(p.h, GS_PIPELINE, 4)


def test_stalled_sweep_times_out_and_the_device_stays_usable():
    """A tile whose predecessors never run: its bounded wait runs out, the
    sweep records the error, the solve returns HPG_ERR_TIMEOUT, and the next
    solve on the same handle is normal (no GPU fault: the waits end)."""
    dims = (80, 80, 80)
    n = 80 ** 3
    with hpg.Problem(*dims, beta=0.5) as p:
        ones = torch.ones(n, dtype=torch.float64, device=DEV)
        b = p.to_natural(p.spmv(p.to_storage(ones)))
        hpg.set_execution(p.h, hpg.HPG_EXEC_EAGER)   # the stall lands in the first V-cycle
        assert hpg.load().hpg_inject_stall(p.h, 0, 1) == hpg.HPG_OK
        x = torch.zeros_like(b)
        info = hpg.gmres_ir_solve(p.h, b, x, tol=1e-9, inner=hpg.HPG_FP64, raise_on_error=False)
        assert info["status"] == hpg.HPG_ERR_TIMEOUT and info["converged"] == 0
        x.zero_()
        info = hpg.gmres_ir_solve(p.h, b, x, tol=1e-9, inner=hpg.HPG_FP64)
        assert info["status"] == 0 and info["converged"] == 1
        assert hpg.load().hpg_inject_stall(p.h, 9, 1) == hpg.HPG_ERR_INVALID
