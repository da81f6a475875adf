"""Parity of hpg_mg_smooth (symmetric multicolour Gauss-Seidel, eqs. (1)-(2),
Sec. 3.2.1) with the oracle's sweeps, through the C ABI."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from oracle import hpg_oracle as O  # noqa: E402
from tests.gpu_helpers import (FP32_REL, FP64_REL, oracle_hierarchy, to_natural,  # noqa: E402
                               to_storage)
from workloads import random_vector  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def oracle_sweeps(L, r, z0, sweeps):
    z = np.zeros(L.n) if z0 is None else z0.copy()
    for _ in range(sweeps):
        O.symgs(L, r, z)
    return z


@pytest.mark.parametrize("dims", [(16, 16, 16), (24, 20, 28), (33, 17, 9)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_smooth_matches_oracle_every_level(dims, dtype):
    lv = oracle_hierarchy(dims, 4, 0.5)
    npdt = np.float64 if dtype == torch.float64 else np.float32
    with hpg.Problem(*dims, beta=0.5, levels=4) as p:
        for l, L in enumerate(lv):
            r = random_vector(L.n, seed=41 + l, dtype=npdt).astype(np.float64)
            z0 = random_vector(L.n, seed=51 + l, dtype=npdt).astype(np.float64)
            for sweeps, zero in [(1, True), (2, True), (1, False), (3, False)]:
                rt = torch.tensor(to_storage(r, L.dims), dtype=dtype, device=DEV)
                if zero:
                    # z enters as 0 and must not be read: fill the rows with NaN
                    init = to_storage(np.full(L.n, np.nan), L.dims)
                else:
                    init = to_storage(z0, L.dims)
                zt = torch.tensor(init, dtype=dtype, device=DEV)
                hpg.mg_smooth(p.h, l, rt, zt, sweeps, zero)
                z = to_natural(zt.cpu().numpy(), L.dims).astype(np.float64)
                ref = oracle_sweeps(L, r, None if zero else z0, sweeps)
                assert np.isfinite(z).all()
                if dtype == torch.float64:
                    assert np.abs(z - ref).max() <= FP64_REL * np.abs(ref).max(), (l, sweeps)
                else:
                    assert np.linalg.norm(z - ref) <= FP32_REL * np.linalg.norm(ref), (l, sweeps)
                # padding rows of the storage order stay 0
                pad = np.ones(zt.numel(), dtype=bool)
                pad[to_storage(np.arange(L.n, dtype=np.float64) + 1, L.dims) > 0] = False
                assert (zt.cpu().numpy()[pad] == 0).all()


def test_smooth_zero_sweeps_and_invalid():
    dims = (8, 8, 8)
    with hpg.Problem(*dims, levels=3) as p:
        r = torch.ones(p.n_store(), dtype=torch.float64, device=DEV)
        z = torch.full_like(r, 3.0)
        hpg.mg_smooth(p.h, 0, r, z, 0, False)
        assert (z == 3.0).all()
        hpg.mg_smooth(p.h, 0, r, z, 0, True)
        assert (z == 0.0).all()
        with pytest.raises(hpg.HpgError):
            hpg.mg_smooth(p.h, 0, r, z, -1, False)
        with pytest.raises(hpg.HpgError):
            hpg.mg_smooth(p.h, 3, r, z, 1, False)
        with pytest.raises(hpg.HpgError):
            hpg.mg_smooth(p.h, 0, r, r, 1, False)


def test_vcycle_pre_smoothing_is_the_smoother():
    """The V-cycle's pre-smoother and hpg_mg_smooth launch the same phases:
    with no coarse correction visible (coarsest level) they agree bitwise."""
    dims = (16, 16, 16)
    with hpg.Problem(*dims, levels=4) as p:
        lvl = 3
        n = p.info[lvl]["n_store"]
        r = torch.randn(n, dtype=torch.float64, device=DEV, generator=torch.Generator(
            device=DEV).manual_seed(3))
        mask = torch.tensor(to_storage(np.ones(p.info[lvl]["n"]), p.info[lvl]["dims"]) > 0,
                            device=DEV)
        r = torch.where(mask, r, torch.zeros_like(r))
        zv = torch.empty_like(r)
        hpg.mg_vcycle(p.h, lvl, r, zv)
        zs = p.smooth(r, level=lvl)
        torch.testing.assert_close(zs, zv, rtol=0, atol=0)
