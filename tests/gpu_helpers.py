"""Helpers of the GPU parity tests: the documented storage layout restated
independently of the library, tolerances, and cached oracle hierarchies."""

import functools

import numpy as np

from oracle import hpg_oracle as O

# Tolerances.  FP64 kernels: 1e-13 relative.  FP32 SpMV: an FMA chain of 27
# terms plus the rounding of the matrix entry to FP32 is bounded elementwise
# by gamma_28 = 28 u / (1 - 28 u) with u = 2^-24, times (|A| |x|)_i.
FP64_REL = 1e-13
FP32_REL = 1e-6
U32 = 2.0 ** -24
FP32_ELEM = 28 * U32 / (1 - 28 * U32)


def colour_block_dims(n):
    """Per colour c: number of coordinates with the colour's parity."""
    out = []
    for c in range(8):
        par = [1 - (c & 1), 1 - ((c >> 1) & 1), 1 - ((c >> 2) & 1)]
        out.append(tuple(max(0, (n[a] - par[a] + 1) // 2) for a in range(3)))
    return out


def storage_layout(dims):
    """(store_index[natural], n_store, offsets) of the colour-blocked order the
    header documents: colour c = ((i+1)&1) + 2((j+1)&1) + 4((k+1)&1), blocks in
    colour order, lexicographic over (i>>1, j>>1, k>>1), 32-row padding."""
    nx, ny, nz = dims
    cd = colour_block_dims(dims)
    offs = [0]
    for c in range(8):
        cnt = cd[c][0] * cd[c][1] * cd[c][2]
        offs.append(offs[-1] + (cnt + 31) // 32 * 32)
    q = np.arange(nx * ny * nz, dtype=np.int64)
    i, j, k = q % nx, (q // nx) % ny, q // (nx * ny)
    c = ((i + 1) & 1) + 2 * ((j + 1) & 1) + 4 * ((k + 1) & 1)
    cdx = np.array([d[0] for d in cd])[c]
    cdy = np.array([d[1] for d in cd])[c]
    idx = np.array(offs)[c] + (i >> 1) + cdx * ((j >> 1) + cdy * (k >> 1))
    return idx, offs[-1], offs


def to_storage(v, dims):
    idx, ns, _ = storage_layout(dims)
    out = np.zeros(ns, dtype=v.dtype)
    out[idx] = v
    return out


def to_natural(v, dims):
    idx, _, _ = storage_layout(dims)
    return v[idx]


@functools.lru_cache(maxsize=16)
def oracle_hierarchy(dims, levels, beta):
    return O.build_hierarchy(*dims, levels=levels, beta=beta)


def abs_matvec(A, x):
    """(|A| |x|): the scale of each entry's rounding error."""
    return abs(A) @ np.abs(x)
