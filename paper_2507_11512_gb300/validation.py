"""Validation phase of the benchmark and its penalty (Sec. 3; the alternative
full-scale validation of Sec. 3.3).

* standard: FP64 GMRES from x0 = 0 converges the relative residual to tol
  (1e-9) within the iteration limit (10,000): n_d inner steps.  Mixed-precision
  GMRES-IR then converges to the same tol: n_ir inner steps.
* fullscale: FP64 GMRES runs until tol or nd_max inner steps, whichever comes
  first; the relative residual it reached is tau.  GMRES-IR then runs until
  its relative residual is below tau: n_ir steps.

The raw GFLOP/s is multiplied by min(1, n_d / n_ir): fewer mixed-precision
steps earn nothing, more are penalised.  On one GPU the validation problem is
the benchmark problem itself (the paper's standard mode validates on one node),
so the two modes differ only in the FP64 iteration cap.
"""

from . import metrics

MODES = ("standard", "fullscale")


def validate(solve, mode="standard", tol=1e-9, nd_max=10000, nir_max=None):
    """Runs the validation phase with `solve(precision, tol, maxit)`, a callable
    that solves from x0 = 0 with "fp64" (Algorithm 2) or "mxp" (Algorithm 3) and
    returns the solve info (iterations, rel_residual, converged, status).
    Returns the phase's record, with the penalty factor."""
    if mode not in MODES:
        raise ValueError("validation mode must be one of %s" % (MODES,))
    if nir_max is None:
        nir_max = 10 * nd_max
    d = solve("fp64", tol, nd_max)
    if d["converged"]:
        tau = tol
    elif mode == "fullscale":
        tau = d["rel_residual"]
    else:
        raise RuntimeError("standard validation: FP64 GMRES did not reach %g in %d steps "
                           "(relative residual %g); use the fullscale mode"
                           % (tol, nd_max, d["rel_residual"]))
    m = solve("mxp", tau, nir_max)
    n_d, n_ir = d["iterations"], m["iterations"]
    return {"mode": mode, "tol": tol, "nd_max": nd_max, "tau": tau, "n_d": n_d, "n_ir": n_ir,
            "fp64_converged": bool(d["converged"]), "mxp_converged": bool(m["converged"]),
            "fp64_rel_residual": d["rel_residual"], "mxp_rel_residual": m["rel_residual"],
            "penalty": metrics.penalty(n_d, n_ir) if m["converged"] else 0.0}
