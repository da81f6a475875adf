"""Many right-hand sides, many systems: thin binding of the library's batch
entry points (argument marshalling only; every step runs in its kernels).

* R-vectors: torch float32 tensors of shape (n_store, R), contiguous, storage
  order of a level (the R values of a row adjacent).
* Right-hand sides and solutions of a solve: torch float64 tensors of shape
  (R, n), natural order.
"""

import ctypes

from . import Problem
from ._lib import HPG_ERR_NOT_CONVERGED, HPG_OK, HpgError, SolveInfo, check, load

KIND_GS, KIND_SPMV = 0, 1


def _ptr(t):
    return t.data_ptr()


def _stream(stream):
    from . import _stream as s
    return s(stream)


def spmv_batch(h, level, X, Y, stream=None):
    """Y = A_level X for the R columns of X (storage-order R-vectors)."""
    check(load().hpg_spmv_batch(h, level, X.shape[1], _ptr(X), _ptr(Y), _stream(stream)),
          "hpg_spmv_batch")


def vcycle_batch(h, level, R, Z, stream=None):
    """Z = M^{-1} R column by column (storage-order R-vectors)."""
    check(load().hpg_mg_vcycle_batch(h, level, R.shape[1], _ptr(R), _ptr(Z), _stream(stream)),
          "hpg_mg_vcycle_batch")


def permute_batch(h, level, direction, nrhs, x_in, x_out, stream=None):
    """float32 R-vectors between natural (R, n) and storage (n_store, R) order."""
    check(load().hpg_permute_batch(h, level, direction, nrhs, _ptr(x_in), _ptr(x_out),
                                   _stream(stream)), "hpg_permute_batch")


def solve_batch(h, B, X, tol=1e-9, restart=30, maxit=10000, stream=None, raise_on_error=True):
    """GMRES-IR for the R right-hand sides B (R, n) float64; X (R, n) holds the
    initial guesses and receives the solutions.  Returns one info dict per
    right-hand side."""
    R = B.shape[0]
    infos = (SolveInfo * R)()
    st = load().hpg_gmres_ir_solve_batch(h, R, _ptr(B), _ptr(X), tol, restart, maxit, infos,
                                         _stream(stream))
    if st not in (HPG_OK, HPG_ERR_NOT_CONVERGED) and raise_on_error:
        raise HpgError(st, "hpg_gmres_ir_solve_batch")
    return [i.as_dict() for i in infos]


def set_shape(h, level, kind, nrhs, lpr, block):
    check(load().hpg_batch_set_shape(h, level, kind, nrhs, lpr, block), "hpg_batch_set_shape")


def get_shape(h, level, kind, nrhs):
    lpr, block = ctypes.c_int(), ctypes.c_int()
    check(load().hpg_batch_get_shape(h, level, kind, nrhs, ctypes.byref(lpr),
                                     ctypes.byref(block)), "hpg_batch_get_shape")
    return lpr.value, block.value


def tune(h, nrhs, stream=None):
    """Autotunes the multi-right-hand-side launch shapes of every level."""
    check(load().hpg_batch_tune(h, nrhs, _stream(stream)), "hpg_batch_tune")


class BatchSolver:
    """Several Problems solved by one CUDA graph launch (hpg_batch_*)."""

    def __init__(self, problems, nrhs, restart=30, tune_shapes=False):
        """tune_shapes: per-problem isolated tuning (hpg_batch_tune) before the
        capture; for the batch itself prefer tune(), which times the batch."""
        self.problems = list(problems)
        self.nrhs = nrhs
        self.restart = restart
        if tune_shapes:
            for p in self.problems:
                tune(p.h, nrhs)
        arr = (ctypes.c_void_p * len(self.problems))(*[p.h for p in self.problems])
        out = ctypes.c_void_p()
        check(load().hpg_batch_create(arr, len(self.problems), nrhs, restart,
                                      ctypes.byref(out)), "hpg_batch_create")
        self.b = out.value

    def solve(self, Bs, Xs, tol=1e-9, maxit=10000, stream=None, raise_on_error=True):
        n = len(self.problems)
        bp = (ctypes.c_void_p * n)(*[_ptr(b) for b in Bs])
        xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in Xs])
        infos = (SolveInfo * (n * self.nrhs))()
        st = load().hpg_batch_solve(self.b, bp, xp, tol, maxit, infos, _stream(stream))
        if st not in (HPG_OK, HPG_ERR_NOT_CONVERGED) and raise_on_error:
            raise HpgError(st, "hpg_batch_solve")
        d = [i.as_dict() for i in infos]
        return [d[i * self.nrhs:(i + 1) * self.nrhs] for i in range(n)]

    def tune(self, Bs, Xs, tol=1e-9, maxit=10000, stream=None):
        """hpg_batch_tune_solve: times whole batch solves of (Bs, Xs) per
        candidate launch shape and keeps the fastest (Xs is overwritten)."""
        n = len(self.problems)
        bp = (ctypes.c_void_p * n)(*[_ptr(b) for b in Bs])
        xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in Xs])
        times = (ctypes.c_float * 3)()
        check(load().hpg_batch_tune_solve(self.b, bp, xp, tol, maxit, times, _stream(stream)),
              "hpg_batch_tune_solve")
        cand = sorted({1, min(2, self.nrhs), self.nrhs})
        return dict(zip(cand, list(times)[:len(cand)]))

    def close(self):
        """Releases the batch's graph.  Close a BatchSolver before its
        Problems: the library refuses to destroy a problem a batch uses."""
        if self.b:
            load().hpg_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def main(argv=None):
    """Times the batched workload: 64 systems, grid edges drawn from
    {24, 32, 48, 64, 96}, nonsymmetric scale sigma ~ U[0.5, 1.5] (beta =
    0.5 sigma), 8 right-hand sides ~ N(0, 1) each, tol 1e-8, seed 0; one graph
    launch solves all of them.  Prints one JSON line."""
    import argparse
    import json
    import time

    import torch

    from . import build, metrics
    import workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=64)
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-tune", action="store_true")
    a = ap.parse_args(argv)
    build.build()
    dev = torch.device("cuda")
    spec = workloads.batch_systems(a.systems, a.nrhs, seed=0)
    t0 = time.perf_counter()
    probs = [Problem(*s["dims"], beta=s["beta"]) for s in spec]
    Bs = [torch.tensor(s["rhs"], dtype=torch.float64, device=dev) for s in spec]
    Xs = [torch.zeros_like(b) for b in Bs]
    setup_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    solver = BatchSolver(probs, a.nrhs)
    tune_ms = None
    if not a.no_tune:
        tune_ms = solver.tune(Bs, Xs, tol=a.tol)
    create_s = time.perf_counter() - t1
    shape = get_shape(probs[0].h, 0, KIND_GS, a.nrhs)
    times, infos = [], None
    for it in range(a.reps + 1):
        for x in Xs:
            x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = solver.solve(Bs, Xs, tol=a.tol)
        e1.record()
        torch.cuda.synchronize()
        if it > 0:
            times.append(e0.elapsed_time(e1))
    ms = sorted(times)[len(times) // 2]
    flops = 0.0
    for s, inf in zip(spec, infos):
        dl = metrics.level_dims(s["dims"], 4)
        for i in inf:
            flops += metrics.solve_flops(dl, metrics.cycles_from_info(i["iterations"],
                                                                      i["restarts"], 30))
    its = [i["iterations"] for inf in infos for i in inf]
    ok = all(i["converged"] for inf in infos for i in inf)
    # byte-model roofline: the library's algorithmic bytes of every launch of
    # each system's batched solve (profiled one system at a time, from x0 = 0;
    # same iterations as in the batch) over the batch solve's time
    from . import profile_report, set_profiling
    total_bytes = 0.0
    for pr, b in zip(probs, Bs):
        x = torch.zeros_like(b)
        set_profiling(pr.h, True)
        solve_batch(pr.h, b, x, tol=a.tol)
        total_bytes += sum(r["bytes"] for r in profile_report(pr.h))
        set_profiling(pr.h, False)
    peak = None
    import json as _json
    import os as _os
    pk = _os.path.join(_os.path.dirname(_os.path.dirname(_os.path.abspath(__file__))),
                       "MEASURED_PEAKS.json")
    if _os.path.exists(pk):
        with open(pk) as f:
            peak = _json.load(f).get("hbm_gbs")
    gbs = total_bytes / (ms / 1e3) / 1e9
    unknowns = sum(s["dims"][0] * s["dims"][1] * s["dims"][2] for s in spec)
    print(json.dumps({
        "workload": "batch_%dsys_%drhs" % (a.systems, a.nrhs), "systems": a.systems,
        "nrhs": a.nrhs, "unknowns": unknowns, "tol": a.tol, "all_converged": ok,
        "ms_per_batch_solve": ms, "gflops": flops / (ms / 1e3) / 1e9,
        "rhs_solved_per_s": a.systems * a.nrhs / (ms / 1e3),
        "iterations_min_median_max": [min(its), sorted(its)[len(its) // 2], max(its)],
        "setup_s": setup_s, "tune_and_capture_s": create_s, "tuned": not a.no_tune,
        "lanes_per_row": shape[0], "tuning_solve_ms_by_lanes_per_row": tune_ms,
        "roofline": {"bound": "hbm", "bytes": total_bytes, "achieved": gbs, "unit": "GB/s",
                     "peak": peak, "frac": gbs / peak if peak else None,
                     "timing": "library per-launch algorithmic bytes of every system's "
                               "batched solve over the batch solve's CUDA-event time"}}))
    solver.close()
    for p in probs:
        p.close()


if __name__ == "__main__":
    main()
