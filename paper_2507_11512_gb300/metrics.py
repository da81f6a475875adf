"""Benchmark accounting of the HPG-MxP solve: flop model, byte model, penalty.

The paper counts floating-point operations "using a carefully constructed
model" with every precision counted equally (Sec. 3) and updates the count
for the fused SpMV-restriction (Sec. 3.2.4) but does not print the model.
This module states one:

* SpMV: 2 flops per structural non-zero;
* Gauss-Seidel half sweep: 2 nnz + n (one divide per row);
* fused residual-restriction: 2 x the non-zeros of the coarse-coincident fine
  rows + n_c (the subtraction from r);
* prolongation: n_c additions;
* CGS2 at inner step k (k+1 basis vectors): 4 passes of 2 n (k+1);
* Arnoldi norm 2n, normalisation n;
* per restart cycle: outer residual 2 nnz + n, its norm 2n, TRSM k^2,
  Q t 2 n k, one V-cycle, x update n;
* one final outer residual and norm.

Non-zeros are the structural ones (padding slots excluded).  Everything is
closed form in the grid dimensions.
"""


def axis_pairs(n):
    return 3 * n - 2 if n >= 1 else 0


def nnz(dims):
    """Structural non-zeros of the 27-point matrix on an nx x ny x nz grid."""
    nx, ny, nz = dims
    return axis_pairs(nx) * axis_pairs(ny) * axis_pairs(nz)


def coarse_point_nnz(dims):
    """Non-zeros of the fine rows at even (coarse-coincident) points: along an
    axis of even length n the even coordinates 0, 2, ..., n-2 have 2, 3, ..., 3
    neighbours within the grid."""
    out = 1
    for n in dims:
        out *= 3 * (n // 2) - 1
    return out


def level_dims(dims, levels):
    out = [tuple(dims)]
    while len(out) < levels and all(d % 2 == 0 for d in out[-1]):
        out.append(tuple(d // 2 for d in out[-1]))
    return out


def vcycle_flops(dims_list, lev=0, pre=1, post=1):
    d = dims_list[lev]
    n = d[0] * d[1] * d[2]
    half = 2 * nnz(d) + n
    if lev == len(dims_list) - 1:
        return 2 * half
    nc = n // 8
    return ((pre + post) * 2 * half + 2 * coarse_point_nnz(d) + nc + nc
            + vcycle_flops(dims_list, lev + 1, pre, post))


def cycles_from_info(iterations, restarts, restart):
    """Inner steps of every restart cycle: full cycles, then the remainder."""
    if restarts <= 0:
        return []
    full = [restart] * (restarts - 1)
    return full + [iterations - restart * (restarts - 1)]


def solve_flops(dims_list, cycles, pre=1, post=1):
    d = dims_list[0]
    n = d[0] * d[1] * d[2]
    z = nnz(d)
    vc = vcycle_flops(dims_list, 0, pre, post)
    total = 0
    for kc in cycles:
        total += 2 * z + n + 2 * n
        for k in range(kc):
            total += vc + 2 * z + 8 * n * (k + 1) + 2 * n + n
        total += kc * kc + 2 * n * kc + vc + n
    total += 2 * z + n + 2 * n
    return total


def penalty(n_d, n_ir):
    """Sec. 3: F = F_raw * n_d / n_ir when that ratio is below 1, else F_raw."""
    if n_ir <= 0:
        return 1.0
    return min(1.0, n_d / n_ir)


def gs_row_bytes(value_bytes, vector_bytes):
    """Algorithmic DRAM bytes of one row of a Gauss-Seidel colour phase: the
    27 ELL values, the 26 off-diagonal int32 indices, r_i, the write of z_i and
    the gathered z_j (each neighbour value read once over the sweep)."""
    return 27 * value_bytes + 26 * 4 + 3 * vector_bytes


def inner_iteration_bytes(dims_list, k, value_bytes, vector_bytes, pre=1, post=1):
    """Algorithmic DRAM bytes of one inner step at basis size k+1 (context)."""
    sv, sx = value_bytes, vector_bytes
    tot = 0.0
    for lev, d in enumerate(dims_list):
        n = d[0] * d[1] * d[2]
        gs_row = gs_row_bytes(sv, sx)
        sweeps = 1 if lev == len(dims_list) - 1 else pre + post
        tot += sweeps * 15 / 8 * n * gs_row
        if lev < len(dims_list) - 1:
            tot += n / 8 * (27 * (sv + 4) + 3 * sx) + n / 8 * 3 * sx
    d = dims_list[0]
    n = d[0] * d[1] * d[2]
    tot += n * (27 * (sv + 4) + 2 * sx)
    tot += n * sx * (3 * (k + 1) + 4) + 2 * n * sx
    return tot
