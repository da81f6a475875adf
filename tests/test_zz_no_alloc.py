"""hpg_mg_vcycle_noalloc: the V-cycle for callers that cannot allocate device
memory when they call (inside a CUDA stream capture, in a real-time loop, or
under a memory-pool policy).  Its coarse-level work vectors live in a static
device array the library declares, so it must give what hpg_mg_vcycle gives.

Both are called through the C ABI on the same inputs, twice in a row (the
shared array keeps the previous call's contents).  This file is collected
last on purpose, and it also passes when run alone.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_11512_gb300 as hpg  # noqa: E402
from paper_2507_11512_gb300 import _lib  # noqa: E402
from tests.gpu_helpers import FP32_REL, FP64_REL, to_natural, to_storage  # noqa: E402
from workloads import random_vector  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def call_noalloc(p, level, r, z):
    lib = _lib.load()
    prec = hpg.HPG_FP64 if r.dtype == torch.float64 else hpg.HPG_FP32
    return lib.hpg_mg_vcycle_noalloc(p.h, level, prec, r.data_ptr(), z.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dims,beta", [((32, 32, 32), 0.5), ((24, 20, 28), 0.0),
                                       ((128, 128, 128), 0.5)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_vcycle_matches_vcycle(dims, beta, dtype):
    with hpg.Problem(*dims, beta=beta) as p:
        for level in range(p.levels):
            info = p.info[level]
            for call in range(2):
                r = random_vector(info["n"], seed=100 * call + level,
                                  dtype=np.float64 if dtype == torch.float64 else np.float32)
                rt = torch.tensor(to_storage(r, info["dims"]), dtype=dtype, device="cuda")
                z_ref = p.vcycle(rt, level)
                z = torch.full_like(rt, float("nan"))
                assert call_noalloc(p, level, rt, z) == hpg.HPG_OK, _lib.load().hpg_last_error()
                torch.cuda.synchronize()
                a = to_natural(z.cpu().numpy(), info["dims"]).astype(np.float64)
                b = to_natural(z_ref.cpu().numpy(), info["dims"]).astype(np.float64)
                if dtype == torch.float64:
                    assert np.abs(a - b).max() <= FP64_REL * np.abs(b).max()
                else:
                    assert np.linalg.norm(a - b) <= FP32_REL * np.linalg.norm(b)


def test_noalloc_vcycle_rejects_oversized_work_space():
    # 2 levels on 320 x 320 x 168: the coarse level's two FP64 vectors need
    # 34.4 MB, more than the 32 MiB array; in FP32 they fit (17.2 MB)
    with hpg.Problem(320, 320, 168, beta=0.5, levels=2) as p:
        n = p.n_store(0)
        r = torch.ones(n, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        assert call_noalloc(p, 0, r, z) == hpg.HPG_ERR_INVALID
        assert b"static array" in _lib.load().hpg_last_error()
        r32 = torch.ones(n, dtype=torch.float32, device="cuda")
        z32 = torch.empty_like(r32)
        assert call_noalloc(p, 0, r32, z32) == hpg.HPG_OK
        ref = p.vcycle(r32)
        torch.cuda.synchronize()
        assert torch.equal(z32, ref)
