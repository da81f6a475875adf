"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module only draws random numbers and names problem sizes; it holds none
of the solver's arithmetic (each side forms b = A x_true + e with its own
matrix).  Vectors are FP64, in natural (lexicographic, x fastest) order.
"""

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple
    beta: float = 0.5          # nonsymmetric option; 0.0 is the symmetric matrix
    levels: int = 4
    restart: int = 30
    tol: float = 1e-9
    maxit: int = 10000
    noise_std: float = 0.0     # b = A*1 + N(0, noise_std^2)
    seed: int = 0
    pre: int = 1
    post: int = 1

    @property
    def n(self):
        return self.dims[0] * self.dims[1] * self.dims[2]


# The paper's benchmark sizes, scaled to one GPU.
WORKLOADS = {
    "fp64_gmres30_16cube": Workload("fp64_gmres30_16cube", (16, 16, 16)),
    "mxp_gmres30_128cube": Workload("mxp_gmres30_128cube", (128, 128, 128),
                                    noise_std=1e-3),
    "mxp_gmres50_320cube": Workload("mxp_gmres50_320cube", (320, 320, 320),
                                    restart=50, noise_std=1e-3),
}


def x_true(n):
    """The known solution of the benchmark right-hand side b = A * 1."""
    return np.ones(n, dtype=np.float64)


def rhs_noise(n, std, seed=0):
    """Gaussian noise e ~ N(0, std^2) added to A * 1 (FP64, seeded PCG64)."""
    if std == 0.0:
        return np.zeros(n, dtype=np.float64)
    return std * np.random.default_rng(seed).standard_normal(n)


def random_vector(n, seed, dtype=np.float64):
    """Standard-normal test vector; FP32 vectors are drawn then rounded."""
    v = np.random.default_rng(seed).standard_normal(n)
    return v.astype(dtype)


BATCH_EDGES = (24, 32, 48, 64, 96)


def batch_systems(nsys=64, nrhs=8, seed=0):
    """The batched workload: nsys systems with cubic grid edges drawn
    uniformly from BATCH_EDGES, a per-system nonsymmetric scale
    sigma ~ U[0.5, 1.5] (beta = 0.5 sigma, so |beta| <= 0.75), and nrhs
    right-hand sides ~ N(0, 1) each, laid out as an (nrhs, n) array in natural
    order.  Seeded PCG64, drawn in system order."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsys):
        e = int(rng.choice(BATCH_EDGES))
        sigma = float(rng.uniform(0.5, 1.5))
        n = e ** 3
        out.append({"dims": (e, e, e), "sigma": sigma, "beta": 0.5 * sigma,
                    "rhs": rng.standard_normal((nrhs, n))})
    return out
