"""HPG-MxP GMRES-IR solve path on one GB300 GPU (sm_103a).

Thin Python binding of the C ABI in ``include/hpgmxp.h``: every function
here marshals arguments and calls the library of the same name
(``hpg_<name>``); every step of the solve runs in the library's CUDA kernels.
Tensors are torch CUDA tensors (device memory) unless a function says
otherwise; the stream defaults to torch's current stream.
"""

import ctypes

from ._lib import (HPG_BF16, HPG_ERR_ALLOC, HPG_ERR_BREAKDOWN, HPG_ERR_CUDA,  # noqa: F401
                   HPG_ERR_INVALID, HPG_ERR_NAN, HPG_ERR_NOT_CONVERGED, HPG_ERR_STATE,
                   HPG_ERR_TIMEOUT, HPG_ERR_UNSUPPORTED, HPG_EXEC_EAGER, HPG_EXEC_GRAPH,
                   HPG_FP16, HPG_FP32,
                   HPG_FP64, HPG_OK, HPG_OPT_COARSE_CLUSTER, HPG_OPT_COARSE_CTA, HPG_OPT_GS_HALO,
                   HPG_OPT_GS_PIPELINE, HPG_OPT_PDL_ROWS,
                   HPG_OPT_PDL, HpgError,
                   KernelStat, LevelDesc, SolveInfo, StencilParams, check, load)

__all__ = ["setup_problem", "build_mg_hierarchy", "num_levels", "level_info", "permute",
           "spmv", "mg_vcycle", "mg_smooth", "gmres_ir_solve", "destroy", "set_profiling", "set_execution",
           "diag_scale_gradient",
           "set_option",
           "profile_report", "Problem", "HpgError",
           "HPG_FP64", "HPG_FP32", "HPG_BF16", "HPG_FP16", "load"]


def _torch():
    import torch
    return torch


def _ptr(a):
    """Device or host address of a torch tensor, numpy array or int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    raise TypeError("expected a tensor, an array or an address, got %r" % type(a))


def _stream(stream):
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _prec_of(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return HPG_FP64
    if t.dtype == torch.float32:
        return HPG_FP32
    raise TypeError("vectors must be float64 or float32, got %s" % t.dtype)


def setup_problem(nx, ny, nz, beta=0.0, theta=None):
    """hpg_setup_problem: returns an opaque handle (int).  theta: optional FP64
    natural-order per-cell diagonal scale (host array or device tensor)."""
    lib = load()
    p = StencilParams(beta, _ptr(theta))
    out = ctypes.c_void_p()
    check(lib.hpg_setup_problem(nx, ny, nz, ctypes.byref(p), ctypes.byref(out)),
          "hpg_setup_problem")
    return out.value


def build_mg_hierarchy(h, levels=4, pre_sweeps=1, post_sweeps=1):
    check(load().hpg_build_mg_hierarchy(h, levels, pre_sweeps, post_sweeps),
          "hpg_build_mg_hierarchy")


def num_levels(h):
    v = ctypes.c_int()
    check(load().hpg_num_levels(h, ctypes.byref(v)), "hpg_num_levels")
    return v.value


def level_info(h, level=0):
    d = LevelDesc()
    check(load().hpg_level_info(h, level, ctypes.byref(d)), "hpg_level_info")
    return {"dims": (d.nx, d.ny, d.nz), "n": d.n, "n_store": d.n_store, "nnz": d.nnz,
            "colour_offset": list(d.colour_offset), "colour_count": list(d.colour_count)}


def permute(h, level, direction, x_in, x_out, stream=None):
    """hpg_permute: direction 0 natural -> storage, 1 storage -> natural."""
    check(load().hpg_permute(h, level, direction, _prec_of(x_in), _ptr(x_in), _prec_of(x_out),
                             _ptr(x_out), _stream(stream)), "hpg_permute")


def spmv(h, level, x, y, stream=None):
    """hpg_spmv: y = A_level x (storage order; precision from the dtype)."""
    p = _prec_of(x)
    if _prec_of(y) != p:
        raise TypeError("x and y must have the same dtype")
    check(load().hpg_spmv(h, level, p, _ptr(x), _ptr(y), _stream(stream)), "hpg_spmv")


def mg_vcycle(h, level, r, z, stream=None):
    """hpg_mg_vcycle: z = M^{-1} r from `level` (storage order)."""
    p = _prec_of(r)
    if _prec_of(z) != p:
        raise TypeError("r and z must have the same dtype")
    check(load().hpg_mg_vcycle(h, level, p, _ptr(r), _ptr(z), _stream(stream)),
          "hpg_mg_vcycle")


def mg_smooth(h, level, r, z, sweeps=1, z_is_zero=False, stream=None):
    """hpg_mg_smooth: `sweeps` symmetric multicolour Gauss-Seidel sweeps on z
    (storage order; z_is_zero: z enters as 0 and is not read)."""
    p = _prec_of(r)
    if _prec_of(z) != p:
        raise TypeError("r and z must have the same dtype")
    check(load().hpg_mg_smooth(h, level, p, _ptr(r), _ptr(z), int(sweeps), 1 if z_is_zero else 0,
                               _stream(stream)), "hpg_mg_smooth")


def gmres_ir_solve(h, b, x, tol=1e-9, restart=30, maxit=10000, inner=HPG_FP32, basis=None,
                   stream=None, raise_on_error=True):
    """hpg_gmres_ir_solve.  b, x: FP64 natural-order vectors (device tensors or
    host arrays / pinned tensors); x holds the initial guess and receives the
    solution.  Returns the solve info as a dict.  HPG_ERR_NOT_CONVERGED never
    raises; other failures raise unless raise_on_error is False."""
    lib = load()
    info = SolveInfo()
    if basis is None:
        basis = inner
    st = lib.hpg_gmres_ir_solve(h, _ptr(b), _ptr(x), tol, restart, maxit, inner, basis,
                                ctypes.byref(info), _stream(stream))
    if st not in (HPG_OK, HPG_ERR_NOT_CONVERGED) and raise_on_error:
        raise HpgError(st, "hpg_gmres_ir_solve")
    d = info.as_dict()
    d["status"] = st
    return d


def diag_scale_gradient(h, lam, x, grad, stream=None):
    """hpg_diag_scale_gradient: grad = dL/dtheta = -26 lam * x for the
    diagonal scales of h's fine grid (FP64, natural order, n entries each)."""
    check(load().hpg_diag_scale_gradient(h, _ptr(lam), _ptr(x), _ptr(grad), _stream(stream)),
          "hpg_diag_scale_gradient")


def set_profiling(h, enable=True):
    """hpg_set_profiling: per-kernel-class CUDA-event timing on/off."""
    check(load().hpg_set_profiling(h, 1 if enable else 0), "hpg_set_profiling")


def set_execution(h, mode):
    """hpg_set_execution: HPG_EXEC_GRAPH (default) or HPG_EXEC_EAGER."""
    check(load().hpg_set_execution(h, mode), "hpg_set_execution")


def set_option(h, option, value):
    """hpg_set_option: HPG_OPT_COARSE_CLUSTER, HPG_OPT_PDL (0 / 1) or
    HPG_OPT_GS_PIPELINE (0 never, 1 FP64 sweeps, 2 always)."""
    check(load().hpg_set_option(h, option, int(value)), "hpg_set_option")


def profile_report(h):
    """hpg_profile_report: list of dicts (name, level, prec, launches,
    total_ms, bytes) aggregated since profiling was enabled; clears them."""
    lib = load()
    cap = 32 * 8 * 4   # kernel classes x levels x precisions
    arr = (KernelStat * cap)()
    cnt = ctypes.c_int()
    check(lib.hpg_profile_report(h, arr, cap, ctypes.byref(cnt)), "hpg_profile_report")
    return [{"name": arr[i].name.decode(), "level": arr[i].level, "prec": arr[i].prec,
             "launches": arr[i].launches, "total_ms": arr[i].total_ms, "bytes": arr[i].bytes}
            for i in range(min(cnt.value, cap))]


def destroy(h):
    if h:
        check(load().hpg_destroy(h), "hpg_destroy")


class Problem:
    """Owns one handle; natural-order helpers around the storage-order calls."""

    def __init__(self, nx, ny, nz, beta=0.0, theta=None, levels=4, pre_sweeps=1,
                 post_sweeps=1):
        self.h = setup_problem(nx, ny, nz, beta, theta)
        build_mg_hierarchy(self.h, levels, pre_sweeps, post_sweeps)
        self.dims = (nx, ny, nz)
        self.levels = num_levels(self.h)
        self.info = [level_info(self.h, l) for l in range(self.levels)]

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_store(self, level=0):
        return self.info[level]["n_store"]

    def to_storage(self, x_nat, level=0, dtype=None):
        torch = _torch()
        out = torch.empty(self.n_store(level), dtype=dtype or x_nat.dtype, device=x_nat.device)
        permute(self.h, level, 0, x_nat, out)
        return out

    def to_natural(self, x_st, level=0, dtype=None):
        torch = _torch()
        out = torch.empty(self.info[level]["n"], dtype=dtype or x_st.dtype, device=x_st.device)
        permute(self.h, level, 1, x_st, out)
        return out

    def spmv(self, x_st, level=0):
        y = _torch().empty_like(x_st)
        spmv(self.h, level, x_st, y)
        return y

    def vcycle(self, r_st, level=0):
        z = _torch().empty_like(r_st)
        mg_vcycle(self.h, level, r_st, z)
        return z

    def smooth(self, r_st, z_st=None, level=0, sweeps=1):
        """Symmetric Gauss-Seidel sweeps on z_st in place (from z = 0 when
        z_st is None); returns z."""
        if z_st is None:
            z = _torch().empty_like(r_st)
            mg_smooth(self.h, level, r_st, z, sweeps, True)
            return z
        mg_smooth(self.h, level, r_st, z_st, sweeps, False)
        return z_st

    def solve(self, b, x=None, **kw):
        torch = _torch()
        if x is None:
            x = torch.zeros_like(b)
        info = gmres_ir_solve(self.h, b, x, **kw)
        return x, info
