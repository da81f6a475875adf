"""Planted mistakes in the oracle must be caught by its pins.

Each test swaps one oracle function for a plausible wrong variant (a dropped
term, a flipped sign, a wrong index) and checks that the independent pin of
``test_oracle_pins`` now fails.  Everything runs on the CPU.
"""

import numpy as np
import scipy.linalg as sla

from oracle import hpg_oracle as O
from tests.test_oracle_pins import dense_stencil, dense_vcycle_operator


def vcycle_matches_dense(dims=(8, 8, 8), levels=3, beta=0.5):
    lv = O.build_hierarchy(*dims, levels=levels, beta=beta)
    Minv = dense_vcycle_operator([l.dims for l in lv], beta)
    r = np.random.default_rng(0).standard_normal(lv[0].n)
    return np.allclose(O.vcycle(lv, r), Minv @ r, rtol=1e-10, atol=1e-10)


def gmres_matches_lu(dims=(8, 8, 8), beta=0.5):
    A, _ = dense_stencil(*dims, beta)
    lv = O.build_hierarchy(*dims, levels=4, beta=beta)
    b = np.random.default_rng(1).standard_normal(lv[0].n)
    x, info = O.gmres_ir(lv, b, tol=1e-12, restart=30, maxit=200)
    x_lu = sla.lu_solve(sla.lu_factor(A), b)
    return info.converged and np.linalg.norm(x - x_lu) < 1e-9 * np.linalg.norm(x_lu)


def test_unmutated_oracle_passes():
    assert vcycle_matches_dense()
    assert gmres_matches_lu()


def test_flipped_defect_sign_is_caught(monkeypatch):
    def bad(level, r, z):
        return -r[level.fc] - level.A[level.fc] @ z   # Fig. 1 printed literally
    monkeypatch.setattr(O, "restrict_residual", bad)
    assert not vcycle_matches_dense()


def test_wrong_injection_points_are_caught(monkeypatch):
    def bad(level, zc, z):
        z[level.fc + 1] += zc                        # odd x instead of even
    monkeypatch.setattr(O, "prolong_add", bad)
    assert not vcycle_matches_dense()


def test_forward_only_smoother_is_caught(monkeypatch):
    monkeypatch.setattr(O, "backward_sweep", O.forward_sweep)
    assert not vcycle_matches_dense()


def test_dropped_diagonal_divide_is_caught(monkeypatch):
    def bad(level, c, r, z):
        rows = level.colour_rows[c]
        z[rows] = (r[rows] - level.A_off_colour[c] @ z) / 26.0
    monkeypatch.setattr(O, "gs_colour_phase", bad)
    # with a constant diagonal of 26 the wrong divide is invisible, so the
    # triangular-solve pin runs on a problem with a theta-scaled diagonal
    lv = O.build_hierarchy(4, 4, 4, 1, 0.0,
                           np.random.default_rng(2).uniform(0.9, 1.1, 64))
    A = lv[0].A.toarray()
    r = np.random.default_rng(3).standard_normal(64)
    z = np.zeros(64)
    O.symgs(lv[0], r, z)
    pts = np.array([(i, j, k) for k in range(4) for j in range(4) for i in range(4)])
    col = np.array([O.colour_of(i, j, k) for (i, j, k) in pts])
    perm = np.argsort(col, kind="stable")
    Ap = A[np.ix_(perm, perm)]
    D, L, U = np.diag(np.diag(Ap)), np.tril(Ap, -1), np.triu(Ap, 1)
    y = sla.solve_triangular(D + L, r[perm], lower=True)
    z1 = sla.solve_triangular(D + U, r[perm] - L @ y, lower=False)
    ref = np.empty(64)
    ref[perm] = z1
    assert not np.allclose(z, ref, rtol=1e-12, atol=1e-12)


def test_givens_sign_error_is_caught(monkeypatch):
    real = O.givens_update

    def bad(H, cs, sn, t, k):
        rho = real(H, cs, sn, t, k)
        t[k + 1] = -t[k + 1]                         # wrong sign of -s_k t_k
        return rho
    monkeypatch.setattr(O, "givens_update", bad)
    # iterative refinement repairs a wrong cycle over later restarts, so the
    # pin that sees the mistake is the single-cycle residual estimate
    lv = O.build_hierarchy(8, 8, 8, 4, 0.5)
    b = np.random.default_rng(5).standard_normal(lv[0].n)
    x, info = O.gmres_ir(lv, b, tol=1e-15, restart=7, maxit=7)
    true = np.linalg.norm(b - lv[0].A @ x) / np.linalg.norm(b)
    assert abs(true - info.history[-1]) > 1e-6


def test_single_gram_schmidt_pass_changes_basis_orthogonality_bound():
    # CGS2 keeps ||Q^T Q - I|| at rounding level; the pin uses 1e-13.  A basis
    # built with one CGS pass on a harder (nonsymmetric, larger) problem loses
    # more orthogonality than that bound allows.
    lv = O.build_hierarchy(16, 16, 16, 4, 0.75)
    A = lv[0].A
    q = np.random.default_rng(4).standard_normal(lv[0].n)
    Q = [q / np.linalg.norm(q)]
    for _ in range(25):
        w = A @ O.vcycle(lv, Q[-1])
        Qm = np.column_stack(Q)
        w = w - Qm @ (Qm.T @ w)
        Q.append(w / np.linalg.norm(w))
    Qm = np.column_stack(Q)
    assert np.abs(Qm.T @ Qm - np.eye(len(Q))).max() > 1e-13


def spectrum_matches(dims=(5, 3, 4)):
    nx, ny, nz = dims
    A = O.build_matrix(nx, ny, nz, 0.0).toarray()
    ev = np.sort(np.linalg.eigvalsh(A))
    j = [1.0 + 2.0 * np.cos(np.pi * np.arange(1, n + 1) / (n + 1)) for n in (nx, ny, nz)]
    ref = np.sort((27.0 - np.einsum("i,j,k->ijk", j[0], j[1], j[2])).ravel())
    return np.allclose(ev, ref, rtol=0, atol=1e-12)


def test_periodic_wrap_instead_of_truncation_is_caught(monkeypatch):
    real_index = O.natural_index
    dims = (5, 3, 4)

    def wrapped(i, j, k, nx, ny):
        return real_index(np.mod(i, nx), np.mod(j, ny), np.mod(k, dims[2]), nx, ny)

    def bad(nx, ny, nz, beta=0.0, theta=None):
        # every neighbour kept, out-of-grid ones wrapped around (a torus)
        n = nx * ny * nz
        ii, jj, kk = O.grid_coords(nx, ny, nz)
        A = np.zeros((n, n))
        for (dx, dy, dz) in O.STENCIL_OFFSETS:
            c = wrapped(ii + dx, jj + dy, kk + dz, nx, ny)
            v = 26.0 if (dx, dy, dz) == (0, 0, 0) else O.off_diagonal_value(dx, dy, dz, beta)
            np.add.at(A, (np.arange(n), c), v)
        import scipy.sparse as sp
        return sp.csr_matrix(A)
    assert spectrum_matches(dims)
    monkeypatch.setattr(O, "build_matrix", bad)
    assert not spectrum_matches(dims)


def test_diagonal_off_by_one_is_caught(monkeypatch):
    real = O.build_matrix

    def bad(nx, ny, nz, beta=0.0, theta=None):
        A = real(nx, ny, nz, beta, theta).tolil()
        A.setdiag(A.diagonal() + 1.0)                # 27 instead of 26
        return A.tocsr()
    monkeypatch.setattr(O, "build_matrix", bad)
    assert not spectrum_matches()


def test_stencil_row_mistakes_are_caught(monkeypatch):
    from tests.test_oracle_pins import stencil_row_dense
    dims, beta = (4, 3, 4), 0.5
    theta = np.linspace(0.9, 1.1, 48)
    A, pts = dense_stencil(*dims, beta, theta)

    def matches():
        return all(np.array_equal(stencil_row_dense(*dims, i, j, k, beta, theta[q]), A[q])
                   for q, (i, j, k) in enumerate(pts))

    assert matches()
    good = O.off_diagonal_value
    # the perturbation taken from the row's point of view (d = x_i - x_j)
    monkeypatch.setattr(O, "off_diagonal_value", lambda dx, dy, dz, b: good(-dx, -dy, -dz, b))
    assert not matches()
    monkeypatch.setattr(O, "off_diagonal_value", good)
    # y and z strides swapped in the natural index
    good_idx = O.natural_index
    monkeypatch.setattr(O, "natural_index", lambda i, j, k, nx, ny: i + ny * (j + nx * k))
    assert not matches()
    monkeypatch.setattr(O, "natural_index", good_idx)
    assert matches()
