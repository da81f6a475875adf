"""Pins of the oracle's differentiable solve (dense adjoint gradients) against
central finite differences of the loss, which need no adjoint at all."""

import numpy as np
import pytest

from oracle import hpg_oracle as O


def loss(nx, ny, nz, b, xt, beta, theta):
    A = O.build_matrix(nx, ny, nz, beta, theta).toarray()
    x = np.linalg.solve(A, b)
    return float((x - xt) @ (x - xt))


@pytest.mark.parametrize("dims,beta", [((4, 4, 4), 0.5), ((5, 4, 3), -0.75), ((4, 4, 4), 0.0)])
def test_adjoint_gradients_match_central_differences(dims, beta):
    n = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(3)
    theta = rng.uniform(0.9, 1.1, n)
    b = rng.standard_normal(n)
    xt = rng.standard_normal(n)
    x, L, gb, gt = O.dense_adjoint_gradients(*dims, b, xt, beta, theta)
    assert abs(L - loss(*dims, b, xt, beta, theta)) <= 1e-12 * L
    h = 1e-6
    for i in rng.choice(n, 6, replace=False):
        e = np.zeros(n)
        e[i] = h
        fd_b = (loss(*dims, b + e, xt, beta, theta) - loss(*dims, b - e, xt, beta, theta)) / (2 * h)
        fd_t = (loss(*dims, b, xt, beta, theta + e) - loss(*dims, b, xt, beta, theta - e)) / (2 * h)
        assert abs(fd_b - gb[i]) <= 1e-6 * (abs(gb).max())
        assert abs(fd_t - gt[i]) <= 1e-6 * (abs(gt).max())


def test_adjoint_of_the_nonsymmetric_matrix_is_beta_flipped():
    # the product's backward solves A(-beta) lambda = g; the oracle transposes
    dims, beta = (4, 5, 3), 0.5
    n = 60
    rng = np.random.default_rng(4)
    theta = rng.uniform(0.9, 1.1, n)
    g = rng.standard_normal(n)
    At = O.build_matrix(*dims, beta, theta).toarray().T
    Am = O.build_matrix(*dims, -beta, theta).toarray()
    assert np.array_equal(At, Am)
    assert np.allclose(np.linalg.solve(At, g), np.linalg.solve(Am, g), rtol=0, atol=1e-12)


def test_planted_mistake_fails_the_pin():
    # using A instead of A^T for the adjoint (a plausible mistake) is caught
    dims, beta = (4, 4, 4), 0.75
    n = 64
    rng = np.random.default_rng(5)
    theta = rng.uniform(0.9, 1.1, n)
    b = rng.standard_normal(n)
    xt = rng.standard_normal(n)
    A = O.build_matrix(*dims, beta, theta).toarray()
    x = np.linalg.solve(A, b)
    wrong = np.linalg.solve(A, 2 * (x - xt))
    _, _, gb, _ = O.dense_adjoint_gradients(*dims, b, xt, beta, theta)
    assert np.abs(wrong - gb).max() > 1e-3 * np.abs(gb).max()
