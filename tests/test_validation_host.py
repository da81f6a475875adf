"""Host logic of the validation phase (Sec. 3 and the full-scale mode of
Sec. 3.3) with a fake solver: no GPU."""

import pytest

from paper_2507_11512_gb300 import validation


def fake_solver(fp64_steps_to_tol, mxp_steps_per_decade, fp64_rate=0.9):
    calls = []

    def solve(prec, tol, maxit):
        calls.append((prec, tol, maxit))
        if prec == "fp64":
            if fp64_steps_to_tol <= maxit:
                return {"iterations": fp64_steps_to_tol, "rel_residual": tol * 0.5,
                        "converged": 1, "status": 0}
            return {"iterations": maxit, "rel_residual": fp64_rate ** maxit, "converged": 0,
                    "status": -3}
        import math
        n = int(math.ceil(-math.log10(tol) * mxp_steps_per_decade))
        return {"iterations": n, "rel_residual": tol * 0.9, "converged": 1, "status": 0}
    return solve, calls


def test_standard_mode_penalty():
    solve, calls = fake_solver(90, 12)
    r = validation.validate(solve, "standard", 1e-9, 10000)
    assert r["tau"] == 1e-9 and r["n_d"] == 90 and r["n_ir"] == 108
    assert r["penalty"] == pytest.approx(90 / 108)
    assert calls == [("fp64", 1e-9, 10000), ("mxp", 1e-9, 100000)]


def test_fewer_mixed_precision_steps_earn_nothing():
    solve, _ = fake_solver(200, 10)
    assert validation.validate(solve, "standard")["penalty"] == 1.0


def test_fullscale_mode_uses_the_residual_fp64_reached():
    solve, calls = fake_solver(5000, 10, fp64_rate=0.9)
    r = validation.validate(solve, "fullscale", 1e-9, nd_max=50)
    assert not r["fp64_converged"] and r["n_d"] == 50
    assert r["tau"] == pytest.approx(0.9 ** 50)
    assert calls[1][0] == "mxp" and calls[1][1] == pytest.approx(0.9 ** 50)
    assert r["penalty"] == pytest.approx(min(1.0, 50 / r["n_ir"]))


def test_standard_mode_requires_fp64_convergence():
    solve, _ = fake_solver(5000, 10)
    with pytest.raises(RuntimeError):
        validation.validate(solve, "standard", 1e-9, nd_max=50)
    with pytest.raises(ValueError):
        validation.validate(solve, "other")
