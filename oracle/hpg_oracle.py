"""Plain FP64 CPU oracle of the HPG-MxP GMRES-IR solve path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, tables or helpers), and it
never reads a value produced by the CUDA path.

Everything here is double precision and written for a reader who checks it
against the paper (arXiv 2507.11512, "Scaling the memory wall using
mixed-precision -- HPG-MxP on an exascale machine"):

* problem: the 27-point stencil of Sec. 2 (HPCG's Poisson problem), diagonal
  26 and off-diagonals -1 (Sec. 3), with boundary rows truncated (Sec. 2,
  "fewer non-zeros"), plus an optional nonsymmetric perturbation (Sec. 3 says
  the option exists but does not define it; reading below);
* smoother: symmetric Gauss-Seidel, eqs. (1)-(2) of Sec. 2, in its one-pass
  "relaxation" form over an independent-set (multicolour) ordering (Sec. 3.2.1);
* multigrid: the two-grid cycle of Fig. 1 applied recursively, injection
  restriction eq. (3), prolongation P = R^T (Sec. 3), residual fused with the
  restriction (Sec. 3.2.4, last equation);
* solver: Algorithm 3 (GMRES-IR with CGS2 and Givens rotations); with every
  step in FP64 it is restarted right-preconditioned GMRES, Algorithm 2.

Readings of places where the paper is silent or garbled (each one also listed
in the design notes of the repository):

* nonsymmetric option: a_ij = -1 + beta * (dx + dy + dz) / 3 with
  d = (x_j - x_i) the grid offset of the neighbour; beta = 0 is the benchmarked
  symmetric matrix.  For |beta| <= 1 every row stays weakly diagonally dominant
  (Sec. 3) and A^T is the same stencil with beta -> -beta.
* optional per-cell diagonal scale theta: a_ii = 26 * theta_i.
* coarse operators: the same stencil re-discretised on the coarse grid (same
  beta, diagonal 26, theta injected: theta_c(I) = theta_f(f_c(I))).
* f_c: coarse point (I, J, K) <-> fine point (2I, 2J, 2K), 0-based.
* colours: colour(i, j, k) = ((i+1) & 1) + 2((j+1) & 1) + 4((k+1) & 1), so the
  coarse-coincident points (all coordinates even) form colour 7.  A forward
  sweep visits colours 0..7, a backward sweep 7..0.  With injection transfer
  operators the coarse-coincident colour must not be the first colour of the
  forward sweep (the last one the symmetric pre-smoother touches): that colour's
  residual is exactly zero after the sweep and its correction would be
  overwritten before any neighbour saw it.
* coarsest level: one symmetric sweep from z = 0.
* Fig. 1 prints the restricted defect as d = -r - A z; the reading is
  d = r - A z (the sign that makes the two-grid cycle a solver for A z = r).
* Givens update of Algorithm 3 (garbled subscripts): apply the old rotations
  j = 1..k-1 to column k, then form the rotation that zeroes H[k+1, k].
* inner test: the Givens estimate rho = |t_{k+1}| against tau * ||b||.
* iteration count: the total number of inner (Arnoldi) steps.

Parity unpinned: the flop model (``level_nnz``, ``vcycle_flops``,
``solve_flops``).  The paper says its flop count is carefully constructed but
does not print it, so nothing outside this file fixes these counts; the tests
only check that the library's closed-form count equals them.

The differentiable solve (``dense_adjoint_gradients``) has no counterpart in
the paper: it is the plain definition of the gradient of a loss through
A(theta) x = b by the adjoint equation, written with dense LAPACK solves for
tiny grids.
"""

import math

import numpy as np
import scipy.sparse as sp

# The 27 stencil offsets, x fastest; index 13 is the centre (0, 0, 0).
STENCIL_OFFSETS = [(dx, dy, dz)
                   for dz in (-1, 0, 1)
                   for dy in (-1, 0, 1)
                   for dx in (-1, 0, 1)]
NUM_COLOURS = 8


# ---------------------------------------------------------------- problem --
def natural_index(i, j, k, nx, ny):
    """Lexicographic (x fastest) row number of grid point (i, j, k)."""
    return i + nx * (j + ny * k)


def grid_coords(nx, ny, nz):
    """Arrays (i, j, k) of every row in natural order."""
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    return idx % nx, (idx // nx) % ny, idx // (nx * ny)


def off_diagonal_value(dx, dy, dz, beta):
    """a_ij for the neighbour at offset d = (dx, dy, dz): -1 + beta*(dx+dy+dz)/3."""
    return -1.0 + beta * (dx + dy + dz) / 3.0


def build_matrix(nx, ny, nz, beta=0.0, theta=None):
    """The 27-point stencil matrix of Sec. 2-3 in natural order, as scipy CSR.

    Row i couples grid point i to every grid point within one step in each of
    x, y, z (itself included); neighbours outside the grid are dropped
    (Dirichlet truncation, the "fewer non-zeros" of boundary rows).
    """
    n = nx * ny * nz
    ii, jj, kk = grid_coords(nx, ny, nz)
    rows, cols, vals = [], [], []
    for (dx, dy, dz) in STENCIL_OFFSETS:
        ni, nj, nk = ii + dx, jj + dy, kk + dz
        ok = ((ni >= 0) & (ni < nx) & (nj >= 0) & (nj < ny)
              & (nk >= 0) & (nk < nz))
        r = np.nonzero(ok)[0]
        c = natural_index(ni[ok], nj[ok], nk[ok], nx, ny)
        if (dx, dy, dz) == (0, 0, 0):
            v = 26.0 * (np.ones(len(r)) if theta is None else theta[r])
        else:
            v = np.full(len(r), off_diagonal_value(dx, dy, dz, beta))
        rows.append(r)
        cols.append(c)
        vals.append(v)
    A = sp.csr_matrix((np.concatenate(vals),
                       (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sort_indices()
    return A


def colour_of(i, j, k):
    """Colour of grid point (i, j, k); all-even points are colour 7."""
    return ((i + 1) & 1) + 2 * ((j + 1) & 1) + 4 * ((k + 1) & 1)


def num_levels(nx, ny, nz, requested):
    """Levels actually built: coarsen while every edge is even."""
    levels = 1
    while levels < requested and nx % 2 == 0 and ny % 2 == 0 and nz % 2 == 0:
        nx, ny, nz = nx // 2, ny // 2, nz // 2
        levels += 1
    return levels


class Level:
    """One multigrid level: matrix, colour sets and the coarse->fine map."""

    def __init__(self, nx, ny, nz, beta, theta):
        self.dims = (nx, ny, nz)
        self.n = nx * ny * nz
        self.beta = beta
        self.theta = theta
        self.A = build_matrix(nx, ny, nz, beta, theta)
        self.diag = self.A.diagonal().copy()
        self.A_off = (self.A - sp.diags(self.diag)).tocsr()
        self.A_off.eliminate_zeros()
        ii, jj, kk = grid_coords(nx, ny, nz)
        colour = colour_of(ii, jj, kk)
        self.colour = colour
        self.colour_rows = [np.nonzero(colour == c)[0]
                            for c in range(NUM_COLOURS)]
        # Off-diagonal rows of each colour, so one colour phase is one product.
        self.A_off_colour = [self.A_off[rows] for rows in self.colour_rows]
        self.fc = None  # coarse -> fine map, set when a coarser level exists


def build_hierarchy(nx, ny, nz, levels=4, beta=0.0, theta=None):
    """Multigrid hierarchy: 2x coarsening per axis, re-discretised stencil."""
    L = num_levels(nx, ny, nz, levels)
    out = [Level(nx, ny, nz, beta, theta)]
    for _ in range(1, L):
        fnx, fny, fnz = out[-1].dims
        cnx, cny, cnz = fnx // 2, fny // 2, fnz // 2
        I, J, K = grid_coords(cnx, cny, cnz)
        fc = natural_index(2 * I, 2 * J, 2 * K, fnx, fny)   # f_c(i)
        out[-1].fc = fc
        ctheta = None if theta is None else out[-1].theta[fc]
        out.append(Level(cnx, cny, cnz, beta, ctheta))
    return out


# --------------------------------------------------------------- smoother --
def gs_colour_phase(level, c, r, z):
    """Relaxation of every row of colour c: z_i <- (r_i - sum_{j!=i} a_ij z_j)/a_ii.

    The rows of one colour are an independent set, so updating them all from
    the same z is the sequential Gauss-Seidel update in any order (Sec. 3.2.1).
    """
    rows = level.colour_rows[c]
    z[rows] = (r[rows] - level.A_off_colour[c] @ z) / level.diag[rows]


def forward_sweep(level, r, z):
    """Forward Gauss-Seidel, eq. (1): colours 0, 1, ..., 7."""
    for c in range(NUM_COLOURS):
        gs_colour_phase(level, c, r, z)


def backward_sweep(level, r, z):
    """Backward Gauss-Seidel, eq. (2): colours 7, 6, ..., 0."""
    for c in reversed(range(NUM_COLOURS)):
        gs_colour_phase(level, c, r, z)


def symgs(level, r, z):
    """One symmetric Gauss-Seidel sweep (eqs. (1)-(2)), in place on z."""
    forward_sweep(level, r, z)
    backward_sweep(level, r, z)


# -------------------------------------------------------------- multigrid --
def restrict_residual(level, r, z):
    """Fused residual + injection restriction (Sec. 3.2.4, last equation):
    r^c_i = r_{f_c(i)} - sum_j A_{f_c(i) j} z_j for every coarse point i."""
    fc = level.fc
    return r[fc] - level.A[fc] @ z


def prolong_add(level, zc, z):
    """z <- z + P zc with P = R^T: z_{f_c(i)} += zc_i (eq. (3) transposed)."""
    z[level.fc] += zc


def vcycle(levels, r, lev=0, pre=1, post=1):
    """z = M^{-1} r: one V-cycle from z = 0 (Fig. 1, applied recursively)."""
    level = levels[lev]
    z = np.zeros(level.n)
    if lev == len(levels) - 1:
        symgs(level, r, z)
        return z
    for _ in range(pre):
        symgs(level, r, z)
    rc = restrict_residual(level, r, z)
    zc = vcycle(levels, rc, lev + 1, pre, post)
    prolong_add(level, zc, z)
    for _ in range(post):
        symgs(level, r, z)
    return z


# ------------------------------------------------------------------ GMRES --
def givens_update(H, cs, sn, t, k):
    """Update the QR factorisation of H[:k+2, :k+1] (Algorithm 3, Givens step).

    Applies the stored rotations 0..k-1 to column k, forms rotation k that
    zeroes H[k+1, k], applies it to t and returns rho = |t[k+1]|.
    """
    for j in range(k):
        hj, hj1 = H[j, k], H[j + 1, k]
        H[j, k] = cs[j] * hj + sn[j] * hj1
        H[j + 1, k] = -sn[j] * hj + cs[j] * hj1
    mu = math.hypot(H[k, k], H[k + 1, k])
    if mu == 0.0:
        cs[k], sn[k] = 1.0, 0.0
    else:
        cs[k], sn[k] = H[k, k] / mu, H[k + 1, k] / mu
    H[k, k] = mu
    H[k + 1, k] = 0.0
    t[k + 1] = -sn[k] * t[k]
    t[k] = cs[k] * t[k]
    return abs(t[k + 1])


def back_substitution(U, y):
    """Solve U x = y for upper-triangular U (the dense TRSM of Algorithm 3)."""
    k = len(y)
    x = np.zeros(k)
    for i in reversed(range(k)):
        x[i] = (y[i] - U[i, i + 1:k] @ x[i + 1:k]) / U[i, i]
    return x


class SolveInfo:
    def __init__(self):
        self.iterations = 0        # total inner (Arnoldi) steps
        self.restarts = 0          # completed restart cycles
        self.converged = False
        self.rel_residual = float("nan")   # final ||b - A x|| / ||b||, FP64
        self.history = []          # rho / rho0 after every inner step
        self.outer_history = []    # true relative residual at every restart


def gmres_ir(levels, b, x0=None, tol=1e-9, restart=30, maxit=10000,
             pre=1, post=1, trace=None):
    """Restarted right-preconditioned GMRES with CGS2 (Algorithm 3, all FP64).

    Returns (x, SolveInfo).  If ``trace`` is a list, every restart cycle
    appends a dict with the raw Hessenberg column data (before rotation), the
    basis and the preconditioned vectors, for the Arnoldi-relation checks.
    """
    A = levels[0].A
    n = levels[0].n
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = SolveInfo()
    rho0 = np.linalg.norm(b)
    if rho0 == 0.0:
        info.converged = True
        info.rel_residual = 0.0
        return np.zeros(n), info
    m = restart
    while True:
        r = b - A @ x
        rho = np.linalg.norm(r)
        info.outer_history.append(rho / rho0)
        if rho / rho0 < tol:
            info.converged = True
            break
        if info.iterations >= maxit:
            break
        Q = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        cs, sn, t = np.zeros(m + 1), np.zeros(m + 1), np.zeros(m + 1)
        Q[:, 0] = r / rho
        t[0] = rho
        cyc = None
        if trace is not None:
            cyc = {"Hraw": np.zeros((m + 1, m)), "Z": np.zeros((n, m))}
        k = 0
        while k < m and rho / rho0 >= tol and info.iterations < maxit:
            z = vcycle(levels, Q[:, k], 0, pre, post)
            w = A @ z
            # CGS2: two classical Gram-Schmidt passes.
            h = Q[:, :k + 1].T @ w
            w = w - Q[:, :k + 1] @ h
            H[:k + 1, k] = h
            h = Q[:, :k + 1].T @ w
            w = w - Q[:, :k + 1] @ h
            H[:k + 1, k] += h
            beta = np.linalg.norm(w)
            H[k + 1, k] = beta
            if beta != 0.0:
                Q[:, k + 1] = w / beta
            if cyc is not None:
                cyc["Hraw"][:, k] = H[:, k]
                cyc["Z"][:, k] = z
            rho = givens_update(H, cs, sn, t, k)
            k += 1
            info.iterations += 1
            info.history.append(rho / rho0)
        y = back_substitution(H[:k, :k], t[:k])
        d = vcycle(levels, Q[:, :k] @ y, 0, pre, post)
        x = x + d
        info.restarts += 1
        if cyc is not None:
            cyc.update(k=k, Q=Q[:, :k + 1].copy(), y=y, t=t[:k + 1].copy(),
                       Hrot=H[:k + 1, :k].copy())
            trace.append(cyc)
    info.rel_residual = np.linalg.norm(b - A @ x) / rho0
    return x, info


# ------------------------------------------------------------- flop model --
def level_nnz(level):
    return level.A.nnz


def vcycle_flops(levels, lev=0, pre=1, post=1):
    """Flops of one V-cycle under the counting model (all precisions equal;
    parity unpinned: the paper does not print its model).

    Gauss-Seidel half sweep: 2 nnz + n (one divide per row);
    fused residual-restriction: 2 nnz of the coarse-coincident fine rows + n_c;
    prolongation: n_c additions.
    """
    level = levels[lev]
    half = 2 * level.A.nnz + level.n
    if lev == len(levels) - 1:
        return 2 * half
    fc_nnz = level.A[level.fc].nnz
    return ((pre + post) * 2 * half + 2 * fc_nnz + len(level.fc)
            + len(level.fc) + vcycle_flops(levels, lev + 1, pre, post))


def solve_flops(levels, inner_steps_per_cycle, pre=1, post=1):
    """Flops of a GMRES-IR solve with the given inner steps in each cycle.

    Per inner step k (0-based, k+1 basis vectors): V-cycle, SpMV (2 nnz),
    CGS2 (4 passes of 2 n (k+1)), norm (2n), scaling (n).  Per cycle: outer
    residual (2 nnz + n), norm (2n), TRSM (k^2), Q t (2 n k), V-cycle,
    x update (n).  One extra outer residual and norm for the final check.
    """
    n = levels[0].n
    nnz = levels[0].A.nnz
    vc = vcycle_flops(levels, 0, pre, post)
    total = 0
    for kc in inner_steps_per_cycle:
        total += 2 * nnz + n + 2 * n
        for k in range(kc):
            total += vc + 2 * nnz + 8 * n * (k + 1) + 2 * n + n
        total += kc * kc + 2 * n * kc + vc + n
    total += 2 * nnz + n + 2 * n
    return total


# ------------------------------------------------------- single-row access --
def stencil_row(nx, ny, nz, i, j, k, beta=0.0, theta_ijk=1.0):
    """One matrix row by plain loops: list of (natural column, value)."""
    row = []
    for (dx, dy, dz) in STENCIL_OFFSETS:
        ni, nj, nk = i + dx, j + dy, k + dz
        if 0 <= ni < nx and 0 <= nj < ny and 0 <= nk < nz:
            if (dx, dy, dz) == (0, 0, 0):
                v = 26.0 * theta_ijk
            else:
                v = off_diagonal_value(dx, dy, dz, beta)
            row.append((natural_index(ni, nj, nk, nx, ny), v))
    return row


# ----------------------------------------------------- differentiable solve --
def dense_adjoint_gradients(nx, ny, nz, b, x_target, beta=0.0, theta=None):
    """x = A(theta)^{-1} b, L = ||x - x_target||^2 and its gradients by the
    adjoint equation, with dense LU solves (tiny grids only).

    dL/dx = 2 (x - x_target); the adjoint lambda solves A^T lambda = dL/dx;
    dL/db = lambda; and since only a_ii = 26 theta_i depends on theta_i,
    dL/dtheta_i = -lambda_i * 26 * x_i.  A^T is formed by transposing A here
    (not by flipping beta), so the transpose reading is checked, not assumed.
    Returns (x, L, dL/db, dL/dtheta).
    """
    n = nx * ny * nz
    if theta is None:
        theta = np.ones(n)
    A = build_matrix(nx, ny, nz, beta, theta).toarray()
    x = np.linalg.solve(A, b)
    r = x - x_target
    L = float(r @ r)
    lam = np.linalg.solve(A.T, 2.0 * r)
    return x, L, lam, -26.0 * lam * x

