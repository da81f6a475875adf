"""The seeded input generators: deterministic, of the documented shapes and
ranges, and the same stream for the oracle side and the CUDA side."""

import numpy as np

from workloads import BATCH_EDGES, WORKLOADS, batch_systems, random_vector, rhs_noise, x_true


def test_benchmark_workloads():
    w = WORKLOADS["mxp_gmres30_128cube"]
    assert w.dims == (128, 128, 128) and w.restart == 30 and w.tol == 1e-9
    assert w.noise_std == 1e-3 and w.levels == 4 and w.n == 128 ** 3
    w = WORKLOADS["mxp_gmres50_320cube"]
    assert w.dims == (320, 320, 320) and w.restart == 50
    assert WORKLOADS["fp64_gmres30_16cube"].noise_std == 0.0


def test_rhs_generators_deterministic():
    assert np.array_equal(x_true(5), np.ones(5))
    assert np.array_equal(rhs_noise(7, 0.0), np.zeros(7))
    a, b = rhs_noise(1000, 1e-3, seed=0), rhs_noise(1000, 1e-3, seed=0)
    assert np.array_equal(a, b) and abs(a.std() - 1e-3) < 2e-4
    v32 = random_vector(100, 3, np.float32)
    assert v32.dtype == np.float32
    assert np.array_equal(v32, random_vector(100, 3).astype(np.float32))


def test_batch_systems_shapes_and_ranges():
    s1 = batch_systems(6, 2, seed=0)
    s2 = batch_systems(6, 2, seed=0)
    assert len(s1) == 6
    for a, b in zip(s1, s2):
        assert a["dims"] == b["dims"] and a["sigma"] == b["sigma"]
        assert np.array_equal(a["rhs"], b["rhs"])
        e = a["dims"][0]
        assert a["dims"] == (e, e, e) and e in BATCH_EDGES
        assert 0.5 <= a["sigma"] <= 1.5 and a["beta"] == 0.5 * a["sigma"]
        assert a["rhs"].shape == (2, e ** 3) and a["rhs"].dtype == np.float64
    assert batch_systems(6, 2, seed=1)[0]["sigma"] != s1[0]["sigma"]
