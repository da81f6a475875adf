"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something fixed independently of it: a
closed form, a brute-force construction on a tiny grid, a LAPACK routine
(dense LU, triangular solves, least squares), an invariant of GMRES, or a
number the paper prints (``tests/golden/paper_values.json``).
"""

import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hpg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ------------------------------------------------ brute-force constructions --
def dense_stencil(nx, ny, nz, beta=0.0, theta=None):
    """Dense 27-point matrix from all pairs of grid points (no stencil loop).

    Two points are coupled when they differ by at most one step along every
    axis (Sec. 2); the diagonal is 26 (times theta) and a coupling at offset
    d = q - p is -1 + beta * (dx + dy + dz) / 3.
    """
    pts = np.array([(i, j, k) for k in range(nz) for j in range(ny)
                    for i in range(nx)], dtype=np.int64)
    d = pts[None, :, :] - pts[:, None, :]          # d[p, q] = q - p
    near = np.abs(d).max(axis=2) <= 1
    A = np.where(near, -1.0 + beta * d.sum(axis=2) / 3.0, 0.0)
    diag = 26.0 * (np.ones(len(pts)) if theta is None else theta)
    np.fill_diagonal(A, diag)
    return A, pts


def colour_sorted_perm(pts):
    """Stable permutation that lists rows colour by colour, colour 0 first."""
    col = np.array([O.colour_of(i, j, k) for (i, j, k) in pts])
    return np.argsort(col, kind="stable"), col


def dense_symgs(A, r, z0, perm):
    """Symmetric Gauss-Seidel, eqs. (1)-(2), as two LAPACK triangular solves
    on the colour-permuted matrix (forward over colours 0..7, then back)."""
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    L = np.tril(Ap, -1)
    U = np.triu(Ap, 1)
    rp = r[perm]
    zp = z0[perm]
    y = sla.solve_triangular(D + L, rp - U @ zp, lower=True)
    z1 = sla.solve_triangular(D + U, rp - L @ y, lower=False)
    out = np.empty_like(z1)
    out[perm] = z1
    return out


def dense_vcycle_operator(dims_list, beta, pre=1, post=1):
    """Dense M^{-1} of the V-cycle by composing dense operators level by level.

    Level l: Z1 = S(I, 0); D = R (I - A Z1); Z2 = Z1 + R^T M_{l+1}^{-1} D;
    Z3 = S applied ``post`` times from Z2 (Fig. 1 with injection R, eq. (3),
    P = R^T).  The coarsest level is one symmetric sweep from zero.
    """
    def S_apply(A, perm, Rhs, Z):
        # one symmetric sweep on every column of Z for right-hand sides Rhs
        return np.column_stack([dense_symgs(A, Rhs[:, c], Z[:, c], perm)
                                for c in range(Rhs.shape[1])])

    def build(level):
        nx, ny, nz = dims_list[level]
        A, pts = dense_stencil(nx, ny, nz, beta)
        perm, _ = colour_sorted_perm(pts)
        n = len(pts)
        I = np.eye(n)
        if level == len(dims_list) - 1:
            return S_apply(A, perm, I, np.zeros((n, n)))
        Z = np.zeros((n, n))
        for _ in range(pre):
            Z = S_apply(A, perm, I, Z)
        cx, cy, cz = dims_list[level + 1]
        R = np.zeros((cx * cy * cz, n))
        for K in range(cz):
            for J in range(cy):
                for Ic in range(cx):
                    row = Ic + cx * (J + cy * K)
                    fine = 2 * Ic + nx * (2 * J + ny * 2 * K)
                    R[row, fine] = 1.0
        Mc = build(level + 1)
        Z = Z + R.T @ (Mc @ (R @ (I - A @ Z)))
        for _ in range(post):
            Z = S_apply(A, perm, I, Z)
        return Z

    return build(0)


# ------------------------------------------------------------------ matrix --
@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 3, 4), (1, 2, 3), (7, 1, 1)])
@pytest.mark.parametrize("beta", [0.0, 0.5, -0.75])
def test_matrix_matches_brute_force(dims, beta):
    A_dense, _ = dense_stencil(*dims, beta)
    A = O.build_matrix(*dims, beta).toarray()
    np.testing.assert_array_equal(A, A_dense)


@pytest.mark.parametrize("n", [1, 2, 4, 9])
def test_nnz_closed_form(n):
    # each axis contributes 3n - 2 (row, column) pairs within one step
    A = O.build_matrix(n, n + 1, n + 2)
    assert A.nnz == (3 * n - 2) * (3 * (n + 1) - 2) * (3 * (n + 2) - 2)


def test_paper_stencil_values():
    g = golden()["stencil"]
    A = O.build_matrix(5, 5, 5, beta=0.0)
    centre = O.natural_index(2, 2, 2, 5, 5)
    row = A.getrow(centre)
    assert row.nnz == g["points"]
    vals = dict(zip(row.indices, row.data))
    assert vals.pop(centre) == g["diagonal"]
    assert set(vals.values()) == {g["off_diagonal"]}


def test_symmetric_and_transpose_flip():
    A0 = O.build_matrix(4, 5, 3, 0.0)
    assert (A0 - A0.T).count_nonzero() == 0
    Ab = O.build_matrix(4, 5, 3, 0.5)
    Am = O.build_matrix(4, 5, 3, -0.5)
    np.testing.assert_allclose((Ab.T - Am).toarray(), 0.0, atol=1e-15)
    # the perturbation is antisymmetric: A(beta) - A(0) = -(A(beta) - A(0))^T
    P = (Ab - A0).toarray()
    np.testing.assert_allclose(P, -P.T, atol=1e-15)
    assert np.abs(P).max() > 0.1


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0])
def test_weak_diagonal_dominance(beta):
    # Sec. 3: sum_{j != i} |a_ij| <= a_ii for every row
    A = O.build_matrix(6, 5, 4, beta).toarray()
    d = np.diag(A)
    off = np.abs(A).sum(axis=1) - np.abs(d)
    assert np.all(off <= d + 1e-12)


def test_interior_row_sum_zero_symmetric():
    A = O.build_matrix(5, 5, 5, 0.0)
    s = A @ np.ones(125)
    interior = O.natural_index(2, 2, 2, 5, 5)
    assert s[interior] == 0.0
    assert np.all(s >= 0.0)


def test_fp32_copy_exact_for_symmetric():
    A = O.build_matrix(4, 4, 4, 0.0)
    np.testing.assert_array_equal(A.data.astype(np.float32).astype(np.float64),
                                  A.data)


# ---------------------------------------------------------------- colouring --
@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 2), (6, 6, 6)])
def test_colouring_is_independent_sets(dims):
    nx, ny, nz = dims
    A, pts = dense_stencil(nx, ny, nz)
    col = np.array([O.colour_of(i, j, k) for (i, j, k) in pts])
    coupled = (A != 0) & ~np.eye(len(pts), dtype=bool)
    same = col[:, None] == col[None, :]
    assert not np.any(coupled & same)
    assert set(col) <= set(range(8))
    if min(dims) >= 2:
        assert len(set(col)) == golden()["colours"]["colours_3d_27pt"]


def test_colouring_2d_analogue_four_colours():
    # Fig. 2: a 9-point stencil on a 2D mesh needs 4 independent sets
    cols = {O.colour_of(i, j, 0) for i in range(6) for j in range(6)}
    assert len(cols) == golden()["colours"]["colours_2d_9pt"]
    for i in range(5):
        for j in range(5):
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    if (di, dj) != (0, 0) and 0 <= i + di and 0 <= j + dj:
                        assert O.colour_of(i, j, 0) != O.colour_of(i + di, j + dj, 0)


def test_coarse_points_are_colour_seven():
    lv = O.build_hierarchy(8, 6, 4, 3)
    fine = lv[0]
    assert np.all(fine.colour[fine.fc] == 7)
    assert len(fine.fc) == np.count_nonzero(fine.colour == 7)


@pytest.mark.parametrize("dims,req,expect", [
    ((16, 16, 16), 4, 4), ((12, 12, 12), 4, 3), ((4, 4, 4), 4, 3),
    ((8, 8, 8), 4, 4), ((24, 24, 24), 4, 4), ((2, 2, 3), 4, 1),
    ((1, 1, 1), 4, 1), ((128, 128, 128), 4, 4), ((320, 320, 320), 4, 4),
    ((16, 16, 16), 2, 2)])
def test_level_count(dims, req, expect):
    assert O.num_levels(*dims, req) == expect


def test_paper_fixes_four_levels():
    assert O.num_levels(320, 320, 320, golden()["multigrid"]["levels"]) == 4


# ----------------------------------------------------------------- smoother --
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_symgs_equals_two_triangular_solves(beta):
    dims = (5, 4, 6)
    lv = O.build_hierarchy(*dims, levels=1, beta=beta)
    A, pts = dense_stencil(*dims, beta)
    perm, _ = colour_sorted_perm(pts)
    rng = np.random.default_rng(1)
    r = rng.standard_normal(lv[0].n)
    z0 = rng.standard_normal(lv[0].n)
    z = z0.copy()
    O.symgs(lv[0], r, z)
    np.testing.assert_allclose(z, dense_symgs(A, r, z0, perm), rtol=1e-13,
                               atol=1e-13)


def test_forward_sweep_from_zero_is_lower_triangular_solve():
    dims = (4, 4, 4)
    lv = O.build_hierarchy(*dims, levels=1, beta=0.5)
    A, pts = dense_stencil(*dims, 0.5)
    perm, _ = colour_sorted_perm(pts)
    Ap = A[np.ix_(perm, perm)]
    r = np.random.default_rng(2).standard_normal(64)
    z = np.zeros(64)
    O.forward_sweep(lv[0], r, z)
    ref = np.empty(64)
    ref[perm] = sla.solve_triangular(np.tril(Ap), r[perm], lower=True)
    np.testing.assert_allclose(z, ref, rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- multigrid --
@pytest.mark.parametrize("dims,levels,beta", [
    ((8, 8, 8), 4, 0.0), ((8, 4, 8), 3, 0.5), ((4, 4, 4), 4, -0.5),
    ((6, 6, 6), 2, 0.5)])
def test_vcycle_equals_dense_composition(dims, levels, beta):
    lv = O.build_hierarchy(*dims, levels=levels, beta=beta)
    dims_list = [l.dims for l in lv]
    Minv = dense_vcycle_operator(dims_list, beta)
    rng = np.random.default_rng(3)
    for _ in range(3):
        r = rng.standard_normal(lv[0].n)
        np.testing.assert_allclose(O.vcycle(lv, r), Minv @ r, rtol=1e-12,
                                   atol=1e-12)


def test_restriction_is_injection_at_even_points():
    lv = O.build_hierarchy(6, 4, 8, 2)
    fine = lv[0]
    nx, ny, _ = fine.dims
    r = np.arange(fine.n, dtype=np.float64)
    rc = O.restrict_residual(fine, r, np.zeros(fine.n))
    cx, cy, cz = lv[1].dims
    for K in range(cz):
        for J in range(cy):
            for I in range(cx):
                assert rc[I + cx * (J + cy * K)] == r[2 * I + nx * (2 * J + ny * 2 * K)]


def test_vcycle_reduces_error_as_solver():
    # the V-cycle as a stationary iteration converges (spectral radius < 1)
    lv = O.build_hierarchy(16, 16, 16, 4, 0.5)
    A = lv[0].A
    x_true = np.random.default_rng(4).standard_normal(lv[0].n)
    b = A @ x_true
    x = np.zeros(lv[0].n)
    errs = []
    for _ in range(8):
        x = x + O.vcycle(lv, b - A @ x)
        errs.append(np.linalg.norm(x - x_true))
    assert errs[-1] < 0.5 * errs[0]


# -------------------------------------------------------------------- GMRES --
@pytest.mark.parametrize("dims,beta", [((4, 4, 4), 0.0), ((8, 8, 8), 0.0),
                                       ((8, 8, 8), 0.5), ((6, 4, 8), -0.5)])
def test_gmres_matches_dense_lu(dims, beta):
    A, _ = dense_stencil(*dims, beta)
    lv = O.build_hierarchy(*dims, levels=4, beta=beta)
    b = np.random.default_rng(5).standard_normal(lv[0].n)
    x, info = O.gmres_ir(lv, b, tol=1e-13, restart=30, maxit=500)
    assert info.converged
    x_lu = sla.lu_solve(sla.lu_factor(A), b)
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-11


def test_exact_solution_ones_16cube():
    lv = O.build_hierarchy(16, 16, 16, 4, 0.5)
    b = lv[0].A @ np.ones(lv[0].n)
    x, info = O.gmres_ir(lv, b, tol=1e-9, restart=30, maxit=300)
    assert info.converged and info.rel_residual < 1e-9
    assert np.abs(x - 1.0).max() < 1e-6
    assert 5 <= info.iterations <= 40


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_arnoldi_relation_and_orthogonality(beta):
    lv = O.build_hierarchy(8, 8, 8, 4, beta)
    A = lv[0].A
    b = np.random.default_rng(6).standard_normal(lv[0].n)
    trace = []
    O.gmres_ir(lv, b, tol=1e-12, restart=12, maxit=12, trace=trace)
    cyc = trace[0]
    k = cyc["k"]
    Q = cyc["Q"]                    # n x (k+1)
    Z = cyc["Z"][:, :k]             # M^{-1} q_j
    Hbar = cyc["Hraw"][:k + 1, :k]
    # A M^{-1} Q_k = Q_{k+1} Hbar_k (right-preconditioned Arnoldi)
    lhs = A @ Z
    np.testing.assert_allclose(lhs, Q @ Hbar, atol=1e-12 * np.abs(lhs).max())
    for j in range(k):
        np.testing.assert_allclose(Z[:, j], O.vcycle(lv, Q[:, j]), rtol=0, atol=0)
    assert np.abs(Q.T @ Q - np.eye(k + 1)).max() < 1e-13


def test_givens_matches_least_squares():
    lv = O.build_hierarchy(8, 8, 8, 4, 0.5)
    b = np.random.default_rng(7).standard_normal(lv[0].n)
    trace = []
    x, info = O.gmres_ir(lv, b, tol=1e-14, restart=10, maxit=10, trace=trace)
    cyc = trace[0]
    rho0 = np.linalg.norm(b)
    for k in range(1, cyc["k"] + 1):
        Hbar = cyc["Hraw"][:k + 1, :k]
        e1 = np.zeros(k + 1)
        e1[0] = rho0
        y, *_ = np.linalg.lstsq(Hbar, e1, rcond=None)
        res = np.linalg.norm(e1 - Hbar @ y)
        assert abs(res / rho0 - info.history[k - 1]) < 1e-11
    k = cyc["k"]
    Hbar = cyc["Hraw"][:k + 1, :k]
    e1 = np.zeros(k + 1)
    e1[0] = rho0
    y, *_ = np.linalg.lstsq(Hbar, e1, rcond=None)
    np.testing.assert_allclose(cyc["y"], y, rtol=0, atol=1e-12 * np.linalg.norm(y))


def test_residual_estimate_equals_true_residual():
    lv = O.build_hierarchy(8, 8, 8, 4, 0.5)
    A = lv[0].A
    b = np.random.default_rng(8).standard_normal(lv[0].n)
    for k in (1, 3, 7):
        x, info = O.gmres_ir(lv, b, tol=1e-15, restart=k, maxit=k)
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert abs(true - info.history[-1]) < 1e-12


def test_rho_monotone_within_cycle():
    lv = O.build_hierarchy(16, 16, 16, 4, 0.5)
    b = np.random.default_rng(9).standard_normal(lv[0].n)
    x, info = O.gmres_ir(lv, b, tol=1e-10, restart=30, maxit=300)
    h = np.array(info.history[:min(30, len(info.history))])
    assert np.all(np.diff(h) <= 1e-15)


def test_zero_rhs_returns_zero():
    lv = O.build_hierarchy(4, 4, 4, 4)
    x, info = O.gmres_ir(lv, np.zeros(64), x0=np.ones(64))
    assert info.converged and info.iterations == 0
    assert np.all(x == 0.0)


def test_lucky_breakdown_single_point():
    # 1x1x1: A = [26] and one symmetric sweep is the exact inverse, so the
    # second Krylov vector vanishes (beta = 0) after one step.
    lv = O.build_hierarchy(1, 1, 1, 4)
    x, info = O.gmres_ir(lv, np.array([3.0]), tol=1e-12)
    assert info.converged and info.iterations == 1
    assert x[0] == pytest.approx(3.0 / 26.0, rel=1e-15)


def test_maxit_stops_without_convergence():
    lv = O.build_hierarchy(16, 16, 16, 4, 0.5)
    b = np.random.default_rng(10).standard_normal(lv[0].n)
    x, info = O.gmres_ir(lv, b, tol=1e-12, restart=5, maxit=7)
    assert not info.converged
    assert info.iterations == 7
    assert info.restarts == 2


def test_warm_start_from_solution():
    lv = O.build_hierarchy(8, 8, 8, 4, 0.5)
    A = lv[0].A
    x_true = np.random.default_rng(11).standard_normal(lv[0].n)
    x, info = O.gmres_ir(lv, A @ x_true, x0=x_true, tol=1e-9)
    assert info.converged and info.iterations == 0


def test_theta_scaled_diagonal_matches_brute_force():
    rng = np.random.default_rng(12)
    theta = rng.uniform(0.9, 1.1, 4 * 3 * 5)
    A_dense, _ = dense_stencil(4, 3, 5, 0.25, theta)
    A = O.build_matrix(4, 3, 5, 0.25, theta).toarray()
    np.testing.assert_array_equal(A, A_dense)
    lv = O.build_hierarchy(4, 4, 4, 2, 0.0, rng.uniform(0.9, 1.1, 64))
    np.testing.assert_array_equal(lv[1].theta, lv[0].theta[lv[0].fc])


# ------------------------------------------------------- spectral closed form --
@pytest.mark.parametrize("dims", [(6, 6, 6), (5, 3, 4)])
def test_spectrum_matches_kronecker_closed_form(dims):
    """beta = 0: the truncated 27-point operator is 27 I - J_x (x) J_y (x) J_z
    with J_n = tridiag(1, 1, 1) of order n (J's diagonal gives the centre
    1*1*1 = 1, its off-diagonals every neighbour), whose eigenvalues are
    1 + 2 cos(pi k / (n + 1)), k = 1..n.  So the spectrum of A is
    {27 - prod_d (1 + 2 cos(pi k_d / (n_d + 1)))}: every value and every
    boundary truncation of the oracle's matrix enters it."""
    nx, ny, nz = dims
    A = O.build_matrix(nx, ny, nz, 0.0).toarray()
    ev = np.sort(np.linalg.eigvalsh(A))
    j = [1.0 + 2.0 * np.cos(np.pi * np.arange(1, n + 1) / (n + 1)) for n in (nx, ny, nz)]
    ref = np.sort((27.0 - np.einsum("i,j,k->ijk", j[0], j[1], j[2])).ravel())
    np.testing.assert_allclose(ev, ref, rtol=0, atol=1e-12)


def test_theta_scaled_operator_nonsingular_12cube():
    """The differentiable-solve operator (a_ii = 26 theta_i, theta ~ U(0.9, 1.1),
    beta = 0.5) has rows that are not diagonally dominant; its 12^3 instance is
    checked by a dense SVD (LAPACK): smallest singular value well away from 0,
    close to the smallest eigenvalue 27 - (1 + 2 cos(pi/13))^3 = 1.539 of the
    unperturbed symmetric operator; the transpose has the same singular values."""
    rng = np.random.default_rng(0)
    theta = rng.uniform(0.9, 1.1, 12 ** 3)
    A = O.build_matrix(12, 12, 12, 0.5, theta).toarray()
    s = np.linalg.svd(A, compute_uv=False)
    lam0 = 27.0 - (1.0 + 2.0 * np.cos(np.pi / 13.0)) ** 3
    assert 0.5 * lam0 < s[-1] < 2.0 * lam0
    assert s[0] / s[-1] < 100.0
    At = O.build_matrix(12, 12, 12, -0.5, theta).toarray()
    np.testing.assert_array_equal(At, A.T)


# ------------------------------------------------------------ single rows --
def stencil_row_dense(nx, ny, nz, i, j, k, beta, theta_ijk):
    """stencil_row as a dense row vector (natural order)."""
    out = np.zeros(nx * ny * nz)
    for c, v in O.stencil_row(nx, ny, nz, i, j, k, beta, theta_ijk):
        assert out[c] == 0.0, "column listed twice"
        out[c] = v
    return out


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 3, 4), (1, 2, 3), (3, 1, 1)])
@pytest.mark.parametrize("beta", [0.0, 0.5, -0.75])
def test_stencil_row_matches_brute_force_every_point(dims, beta):
    # every point of small grids (interior, faces, edges, corners) against the
    # all-pairs construction, with a per-cell diagonal scale theta != 1
    theta = np.random.default_rng(3).uniform(0.9, 1.1, dims[0] * dims[1] * dims[2])
    A, pts = dense_stencil(*dims, beta, theta)
    for q, (i, j, k) in enumerate(pts):
        row = stencil_row_dense(*dims, i, j, k, beta, theta[q])
        np.testing.assert_array_equal(row, A[q])


def test_stencil_row_matches_matrix_rows_on_a_larger_grid():
    # the rows the full-size GPU tests sample (corners, faces, edges, random
    # interior points) on a grid too large for a dense matrix
    dims, beta = (33, 17, 24), 0.5
    nx, ny, nz = dims
    theta = np.random.default_rng(4).uniform(0.9, 1.1, nx * ny * nz)
    A = O.build_matrix(*dims, beta, theta).tocsr()
    rng = np.random.default_rng(5)
    pts = [tuple(int(v) for v in rng.integers(0, (nx, ny, nz))) for _ in range(200)]
    pts += [(a, b, c) for a in (0, nx - 1) for b in (0, ny - 1) for c in (0, nz - 1)]
    pts += [(0, 5, 7), (nx - 1, 5, 7), (4, 0, 7), (4, ny - 1, 7), (4, 5, 0), (4, 5, nz - 1),
            (0, 0, 9), (nx - 1, ny - 1, 9), (0, 8, nz - 1), (16, 0, 0)]
    for (i, j, k) in pts:
        q = O.natural_index(i, j, k, nx, ny)
        row = O.stencil_row(nx, ny, nz, i, j, k, beta, theta[q])
        ref = A.getrow(q)
        assert sorted(c for c, _ in row) == sorted(ref.indices.tolist())
        got = dict(row)
        for c, v in zip(ref.indices, ref.data):
            assert got[c] == v
        # the row's length is the product of the in-grid neighbours per axis
        per_axis = [sum(1 for d in (-1, 0, 1) if 0 <= p + d < n)
                    for p, n in zip((i, j, k), dims)]
        assert len(row) == per_axis[0] * per_axis[1] * per_axis[2]
