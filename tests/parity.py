"""Comparison helpers for CUDA-vs-oracle parity tests.

Bounds are compared scale-normalised per output row: the error of row r is
max_k |gpu - oracle| / S_r with S_r = max_k max(|lo_r(k)|, |hi_r(k)|) taken
from the oracle; a row whose oracle bounds are all exactly zero must be
exactly zero on the GPU as well.
"""
import numpy as np


def bound_error(got, ref):
    worst = 0.0
    for r in range(ref["hi"].shape[0]):
        S = max(np.max(np.abs(ref["lo"][r])), np.max(np.abs(ref["hi"][r])))
        if S == 0.0:
            assert np.all(got["lo"][r] == 0.0) and np.all(got["hi"][r] == 0.0), f"row {r}: expected exact zeros"
            continue
        e = max(np.max(np.abs(got["lo"][r] - ref["lo"][r])), np.max(np.abs(got["hi"][r] - ref["hi"][r]))) / S
        worst = max(worst, e)
    return worst


def krylov_error(got, ref, j):
    """Relative error of the valid part of H and of P for column j."""
    mu = int(ref["used"][j])
    assert int(got["m_used"][j]) == mu, (int(got["m_used"][j]), mu)
    if mu == 0:
        return 0.0, 0.0
    Hr = ref["H"][j][: mu + 1, :mu]
    Hg = got["H"][j][: mu + 1, :mu]
    eh = np.max(np.abs(Hg - Hr)) / max(np.max(np.abs(Hr)), 1e-300)
    Pr = ref["P"][j][:, :mu]
    Pg = got["P"][j][:, :mu]
    sp = np.max(np.abs(Pr))
    if sp == 0.0:
        assert np.all(Pg == 0.0)
        ep = 0.0
    else:
        ep = np.max(np.abs(Pg - Pr)) / sp
    return eh, ep


def check_violation(got, ref, problem, tol):
    """Identical first violation step and row; counter-example vertex equal
    wherever the basis entry is not negligible."""
    assert got["viol_step"] == ref["viol_step"], (got["viol_step"], ref["viol_step"])
    assert got["viol_row"] == ref["viol_row"]
    if ref["viol_step"] < 0:
        return
    k, r = ref["viol_step"], ref["viol_row"]
    S = max(np.max(np.abs(ref["hi"][r])), 1e-300)
    assert abs(got["ystar"] - ref["ystar"]) <= tol * S
    pmax = max(abs(ref["basis"][j][r, k]) for j in ref["basis"])
    for j in range(problem.i):
        if abs(ref["basis"][j][r, k]) > 1e-9 * pmax:
            assert got["zstar"][j] == ref["zstar"][j]


def margin_ok(ref, problem, rel=1e-7):
    """The violation decision is unambiguous: hi is not within rel * S of
    theta at the violating step or the step before it."""
    if ref["viol_step"] < 0:
        return True
    k, r = ref["viol_step"], ref["viol_row"]
    S = max(np.max(np.abs(ref["hi"][r])), 1e-300)
    th = problem.theta[r]
    ok = abs(ref["hi"][r, k] - th) > rel * S
    if k > 0:
        ok = ok and abs(ref["hi"][r, k - 1] - th) > rel * S
    return ok
