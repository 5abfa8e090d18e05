"""Per-step LP for polyhedral initial and unsafe sets -- TEST INFRASTRUCTURE.

Only the tests may import this module; the product library shares no code
with it.

Sec. 2.1 checks safety with one LP per step t_k = k dt: a state x0 of the
initial set whose image x = e^{A t_k} x0 lies in the unsafe set.  With the
output space y = C x (Sec. 3.1) and the initial space x0 = E z (Sec. 3.2) the
step-k LP works on the o x i basis matrix B_k = C e^{A t_k} E only:

    find z  with  I_z z <= iota  (and the columns' boxes lo <= z <= hi)
            and   U_y B_k z <= upsilon.

Reading (for a result that is unique where the feasibility problem is not):
the LP is asked for its optimal value

    t*_k = min_{z in initial set} max_u (U_u B_k z - upsilon_u) / ||U_u||,

the largest normalised violation of the unsafe constraints that the initial
set can reduce to; the unsafe set is reachable at step k iff t*_k <= tol, and
the minimiser z* is a counter-example there.  For one unsafe row t*_k is the
signed distance, in output units, from the reachable output interval to the
half-space.  Each step's LP is solved by scipy's HiGHS (a library routine).
"""
from __future__ import annotations

import warnings
from typing import Dict, Optional

import numpy as np
from scipy.optimize import OptimizeWarning, linprog

OPTIMAL, UNBOUNDED, EMPTY = 0, 1, 2  # UNBOUNDED: t*_k = -inf; EMPTY: no initial state

# HiGHS by default drops matrix entries below 1e-9 and stops at 1e-7
# feasibility, which moves t* by ~1e-9 when B_k is small (seen against
# brute-force vertex enumeration); the oracle keeps every entry above 1e-12,
# solves without presolve and to 1e-10 feasibility.
HIGHS_OPTIONS = {"presolve": False, "small_matrix_value": 1e-12, "primal_feasibility_tolerance": 1e-10,
                 "dual_feasibility_tolerance": 1e-10}


def normalise(U: np.ndarray, v: np.ndarray):
    """Unsafe rows scaled to unit norm (the same half-spaces)."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    nr = np.linalg.norm(U, axis=1)
    if np.any(nr == 0.0):
        raise ValueError("an unsafe row is zero")
    return U / nr[:, None], v / nr


def step_lp(B: np.ndarray, zlo, zhi, U, v, Iz=None, iota=None):
    """The step LP for one o x i basis matrix B (Sec. 2.1 with the projections
    of Sec. 3.1-3.2): returns (status, t*, z*)."""
    o, i = B.shape
    Un, vn = normalise(U, v)
    rows = [np.hstack([Un @ B, -np.ones((Un.shape[0], 1))])]
    rhs = [vn]
    if Iz is not None and len(Iz):
        Iz = np.atleast_2d(np.asarray(Iz, dtype=np.float64))
        rows.append(np.hstack([Iz, np.zeros((Iz.shape[0], 1))]))
        rhs.append(np.asarray(iota, dtype=np.float64).reshape(-1))
    c = np.zeros(i + 1)
    c[i] = 1.0
    bounds = [(float(zlo[j]), float(zhi[j])) for j in range(i)] + [(None, None)]
    with warnings.catch_warnings():  # small_matrix_value reaches HiGHS as a raw option
        warnings.simplefilter("ignore", OptimizeWarning)
        res = linprog(c, A_ub=np.vstack(rows), b_ub=np.concatenate(rhs), bounds=bounds, method="highs",
                      options=HIGHS_OPTIONS)
    if res.status == 2:
        return EMPTY, np.nan, np.full(i, np.nan)
    if res.status == 3:
        return UNBOUNDED, -np.inf, np.full(i, np.nan)
    if res.status != 0:
        raise RuntimeError(f"linprog: {res.message}")
    x = _vertex(np.vstack(rows), np.concatenate(rhs), bounds, np.asarray(res.x))
    return OPTIMAL, float(x[i]), x[:i]


def _vertex(A, b, bounds, x):
    """HiGHS stops at 1e-10 feasibility; an optimum of an LP is attained at a
    vertex, the solution of its active constraints, so the oracle solves the
    constraints active at HiGHS's point (rows within 1e-8 of equality and
    bounds within 1e-9) as a linear system.  The vertex replaces HiGHS's
    point when it is feasible to 1e-12 and no worse; t is then recomputed
    from z as max_u (U_u B z - upsilon_u), i.e. the last column of A."""
    n = len(x)
    rows, rhs = [], []
    for r in range(len(b)):
        if abs(b[r] - A[r] @ x) <= 1e-8 * (1.0 + abs(b[r])):
            rows.append(A[r])
            rhs.append(b[r])
    for j, (lo, hi) in enumerate(bounds):
        for bd in (lo, hi):
            if bd is not None and abs(x[j] - bd) <= 1e-9 * (1.0 + abs(bd)):
                e = np.zeros(n)
                e[j] = 1.0
                rows.append(e)
                rhs.append(bd)
    if len(rows) < n:
        return x
    M, r = np.array(rows), np.array(rhs)
    if np.linalg.matrix_rank(M) < n:
        return x
    y = np.linalg.lstsq(M, r, rcond=None)[0]
    z = y[:-1].copy()
    for j, (lo, hi) in enumerate(bounds[:-1]):
        if lo is not None:
            z[j] = max(z[j], lo)
        if hi is not None:
            z[j] = min(z[j], hi)
    unsafe = A[:, -1] != 0.0   # rows with the t coefficient
    t = float(np.max(A[unsafe, :-1] @ z - b[unsafe]))
    y = np.append(z, t)
    if np.all(A @ y <= b + 1e-12 * (1.0 + np.abs(b))) and t <= x[-1] + 1e-9:
        return y
    return x


def check(basis_all, zlo, zhi, U, v, Iz=None, iota=None, tol: float = 0.0) -> Dict:
    """Every step of a basis [j][r][k] (i x o x (steps+1)): margins t*_k,
    statuses, minimisers; the first step with t*_k <= tol (or -inf), its z*
    and y* = B_k z*."""
    basis_all = np.asarray(basis_all)
    i, o, S = basis_all.shape
    margin = np.empty(S)
    status = np.empty(S, dtype=np.int32)
    zs = np.empty((S, i))
    for k in range(S):
        status[k], margin[k], zs[k] = step_lp(basis_all[:, :, k].T, zlo, zhi, U, v, Iz, iota)
    hit = [k for k in range(S) if status[k] == UNBOUNDED or (status[k] == OPTIMAL and margin[k] <= tol)]
    viol = hit[0] if hit else -1
    out = {"margin": margin, "status": status, "z": zs, "viol_step": viol, "z_star": None, "y_star": None}
    if viol >= 0 and status[viol] == OPTIMAL:
        out["z_star"] = zs[viol]
        out["y_star"] = basis_all[:, :, viol].T @ zs[viol]
    return out


def feasible(B, zlo, zhi, U, v, Iz, iota, z, tol: float) -> bool:
    """z is in the initial set and B z within tol of the unsafe set."""
    z = np.asarray(z)
    if np.any(z < np.asarray(zlo) - tol) or np.any(z > np.asarray(zhi) + tol):
        return False
    if Iz is not None and len(Iz) and np.any(np.asarray(Iz) @ z > np.asarray(iota) + tol):
        return False
    Un, vn = normalise(U, v)
    return bool(np.all(Un @ (B @ z) <= vn + tol))
