"""ctypes loader of the in-tree CUDA library ``libhpgmxp.so``.

There is no fallback: if the library is missing or fails to load, importing
the package raises, so no GPU call can silently run anything else.
"""

import ctypes
import os

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "libhpgmxp.so")

HPG_OK = 0
HPG_ERR_INVALID = -1
HPG_ERR_CUDA = -2
HPG_ERR_NOT_CONVERGED = -3
HPG_ERR_BREAKDOWN = -4
HPG_ERR_NAN = -5
HPG_ERR_ALLOC = -6
HPG_ERR_STATE = -7
HPG_ERR_UNSUPPORTED = -8
HPG_ERR_TIMEOUT = -9

HPG_FP64, HPG_FP32, HPG_BF16, HPG_FP16 = 0, 1, 2, 3
HPG_EXEC_GRAPH, HPG_EXEC_EAGER = 0, 1
HPG_OPT_COARSE_CLUSTER, HPG_OPT_PDL, HPG_OPT_GS_PIPELINE, HPG_OPT_GS_HALO = 1, 2, 3, 4
HPG_OPT_COARSE_CTA, HPG_OPT_PDL_ROWS = 5, 6


class StencilParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("theta", ctypes.c_void_p)]


class LevelDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("n", ctypes.c_int64), ("n_store", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("colour_offset", ctypes.c_int64 * 9), ("colour_count", ctypes.c_int64 * 8)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("rho0", ctypes.c_double),
                ("kernel_launches", ctypes.c_int), ("graph_launches", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("level", ctypes.c_int), ("prec", ctypes.c_int),
                ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); every function the header declares
SIGNATURES = {
    "hpg_setup_problem": (_I, [_I, _I, _I, ctypes.POINTER(StencilParams), ctypes.POINTER(_P)]),
    "hpg_build_mg_hierarchy": (_I, [_P, _I, _I, _I]),
    "hpg_num_levels": (_I, [_P, ctypes.POINTER(_I)]),
    "hpg_level_info": (_I, [_P, _I, ctypes.POINTER(LevelDesc)]),
    "hpg_permute": (_I, [_P, _I, _I, _I, _P, _I, _P, _P]),
    "hpg_spmv": (_I, [_P, _I, _I, _P, _P, _P]),
    "hpg_mg_vcycle": (_I, [_P, _I, _I, _P, _P, _P]),
    "hpg_mg_smooth": (_I, [_P, _I, _I, _P, _P, _I, _I, _P]),
    "hpg_mg_vcycle_noalloc": (_I, [_P, _I, _I, _P, _P, _P]),
    "hpg_gmres_ir_solve": (_I, [_P, _P, _P, _D, _I, _I, _I, _I, ctypes.POINTER(SolveInfo), _P]),
    "hpg_spmv_batch": (_I, [_P, _I, _I, _P, _P, _P]),
    "hpg_mg_vcycle_batch": (_I, [_P, _I, _I, _P, _P, _P]),
    "hpg_permute_batch": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "hpg_gmres_ir_solve_batch": (_I, [_P, _I, _P, _P, _D, _I, _I, ctypes.POINTER(SolveInfo),
                                      _P]),
    "hpg_batch_set_shape": (_I, [_P, _I, _I, _I, _I, _I]),
    "hpg_batch_get_shape": (_I, [_P, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "hpg_batch_tune": (_I, [_P, _I, _P]),
    "hpg_batch_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, ctypes.POINTER(_P)]),
    "hpg_batch_solve": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I,
                             ctypes.POINTER(SolveInfo), _P]),
    "hpg_batch_destroy": (_I, [_P]),
    "hpg_batch_tune_solve": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I,
                                  ctypes.POINTER(ctypes.c_float), _P]),
    "hpg_set_profiling": (_I, [_P, _I]),
    "hpg_set_execution": (_I, [_P, _I]),
    "hpg_set_option": (_I, [_P, _I, _I]),
    "hpg_inject_stall": (_I, [_P, _I, _I]),
    "hpg_profile_report": (_I, [_P, ctypes.POINTER(KernelStat), _I, ctypes.POINTER(_I)]),
    "hpg_destroy": (_I, [_P]),
    "hpg_diag_scale_gradient": (_I, [_P, _P, _P, _P, _P]),
    "hpg_status_string": (ctypes.c_char_p, [_I]),
    "hpg_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path=LIB_PATH):
    """Loads the library (once) and declares every signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libhpgmxp.so not found at %s; run __graft_entry__.build() "
                          "(or python -m paper_2507_11512_gb300.build)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HpgError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.hpg_last_error().decode()
        super().__init__("%s: %s %s" % (where, lib.hpg_status_string(status).decode(), msg))
        self.status = status


def check(status, where):
    if status != HPG_OK:
        raise HpgError(status, where)
    return status
