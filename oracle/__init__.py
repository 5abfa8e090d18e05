"""CPU oracle for the projected Krylov verification path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline``
/ ``--impl reference`` legs may import this package.  The product library never
loads it and shares no code with it.

The arithmetic lives in ``kv_oracle.c`` (plain FP64 C, optionally OpenMP);
this module compiles it with gcc, marshals numpy arrays through ctypes, and
strings the steps together in the paper's order:

  1. fold b into the dynamics with a constant-1 variable (Sec. 2.1);
  2. for every column E_j of the initial space (Sec. 3.2): beta0 = ||E_j||,
     v1 = E_j / beta0, then Lanczos (symmetric A, Alg. 3/4) or Arnoldi (Alg. 1)
     with P = C V accumulated in the loop (Sec. 3.1, Alg. 4);
  3. basis[j][r][k] = beta0 * P[r,:] e^{H t_k} e_1 (Eq. approx-formula);
  4. box-initial-set output interval, first violation, counter-example vertex
     (the per-step LP of Sec. 2.1 in closed form).

With an error target (Alg. 2 / Alg. 4) the Krylov dimension of a column is the
first of 4, ceil(1.1 k), ... below krylov_m whose Lemma-1 bound (Sec. 4.2) is
below the target, else krylov_m; the bound at the dimension used is reported
either way.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkvoracle.so")
_lock = threading.Lock()
_lib = None

BREAKDOWN_REL = 1e-12


def build(force: bool = False) -> str:
    """Compile kv_oracle.c into oracle/_build/libkvoracle.so (gcc, -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Op(C.Structure):
    _fields_ = [("kind", C.c_int), ("ndim", C.c_int), ("dims", C.c_int64 * 3),
                ("coef", C.c_double), ("h", C.c_double * 3), ("n", C.c_int64),
                ("rp", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("b", C.c_void_p), ("aug", C.c_int), ("trans", C.c_int), ("face", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.ora_num_threads.restype = C.c_int
            lib.ora_dim.restype = C.c_int64
            lib.ora_dim.argtypes = [C.POINTER(_Op)]
            lib.ora_apply.argtypes = [C.POINTER(_Op), P, P]
            for f in (lib.ora_lanczos, lib.ora_arnoldi):
                f.restype = C.c_int
                f.argtypes = [C.POINTER(_Op), P, C.c_int, C.c_int, P, P, P, P, P]
            lib.ora_expm.argtypes = [C.c_int, P, P]
            lib.ora_basis.argtypes = [C.c_int, C.c_int, P, C.c_int, P, C.c_double, C.c_double,
                                      C.c_int, P]
            lib.ora_set_threads.argtypes = [C.c_int]
            lib.ora_lemma1.restype = C.c_double
            lib.ora_lemma1.argtypes = [C.c_int, C.c_int, P, C.c_double, C.c_double, C.c_double, C.c_int]
            lib.ora_bounds.restype = C.c_int
            lib.ora_bounds.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P,
                                       C.POINTER(C.c_int), C.POINTER(C.c_int), P,
                                       C.POINTER(C.c_double)]
            _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's loops from now on."""
    _load().ora_set_threads(int(n))


def num_threads() -> int:
    return int(_load().ora_num_threads())


class _OpHolder:
    """Keeps the numpy arrays referenced by an ora_op alive."""

    def __init__(self, system, aug: bool, trans: bool = False):
        self.keep = []
        op = _Op()
        if hasattr(system, "dims"):
            op.kind = 0
            op.ndim = len(system.dims)
            for a in range(3):
                op.dims[a] = int(system.dims[a]) if a < op.ndim else 1
                op.h[a] = float(system.h[a]) if a < op.ndim else 1.0
            op.coef = float(system.coef)
            op.n = int(np.prod(system.dims, dtype=np.int64))
            face = getattr(system, "face", None)
            if face is not None:
                ff = np.ascontiguousarray(face, dtype=np.float64)
                assert ff.shape == (2 * op.ndim,)
                self.keep.append(ff)
                op.face = _p(ff)
        else:
            op.kind = 1
            op.n = int(system.n)
            rp = np.ascontiguousarray(system.row_ptr, dtype=np.int64)
            col = np.ascontiguousarray(system.col, dtype=np.int32)
            val = np.ascontiguousarray(system.val, dtype=np.float64)
            self.keep += [rp, col, val]
            op.rp, op.col, op.val = _p(rp), _p(col), _p(val)
        b = getattr(system, "b", None)
        if b is not None:
            b = np.ascontiguousarray(b, dtype=np.float64)
            self.keep.append(b)
            op.b = _p(b)
        op.aug = 1 if aug else 0
        op.trans = 1 if trans else 0
        self.op = op

    @property
    def N(self) -> int:
        return int(self.op.n) + int(self.op.aug)


def apply(system, x: np.ndarray, aug: bool = False, trans: bool = False) -> np.ndarray:
    """y = A x (or A' x with the constant variable appended when aug; the
    transposes with trans)."""
    h = _OpHolder(system, aug, trans)
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (h.N,)
    y = np.empty(h.N)
    _load().ora_apply(C.byref(h.op), _p(x), _p(y))
    return y


def _c_arrays(C_row_ptr, C_col, C_val):
    return (np.ascontiguousarray(C_row_ptr, dtype=np.int64),
            np.ascontiguousarray(C_col, dtype=np.int64),
            np.ascontiguousarray(C_val, dtype=np.float64))


def krylov(system, v1: np.ndarray, m: int, C_row_ptr, C_col, C_val, *, method: str,
           aug: bool = False, trans: bool = False):
    """Lanczos (Alg. 3/4) or Arnoldi (Alg. 1) from the normalised v1, on A
    (A' when aug; their transposes when trans).
    Returns (H (m+1) x m, P o x m, number of valid columns)."""
    h = _OpHolder(system, aug, trans)
    v1 = np.ascontiguousarray(v1, dtype=np.float64)
    assert v1.shape == (h.N,)
    crp, ccol, cval = _c_arrays(C_row_ptr, C_col, C_val)
    o = len(crp) - 1
    H = np.zeros((m + 1, m))
    P = np.zeros((o, m))
    f = _load().ora_lanczos if method == "lanczos" else _load().ora_arnoldi
    used = f(C.byref(h.op), _p(v1), m, o, _p(crp), _p(ccol), _p(cval), _p(H), _p(P))
    return H, P, int(used)


def expm(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    m = A.shape[0]
    E = np.empty_like(A)
    _load().ora_expm(m, _p(A), _p(E))
    return E


def basis(H: np.ndarray, P: np.ndarray, used: int, beta0: float, dt: float, steps: int) -> np.ndarray:
    """o x (steps+1): beta0 * P[:, :used] e^{H_used t_k} e_1 for t_k = k dt."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    o = P.shape[0]
    out = np.zeros((o, steps + 1))
    if used == 0 or o == 0:
        return out
    _load().ora_basis(used, H.shape[1], _p(H), o, _p(P), float(beta0), float(dt), steps, _p(out))
    return out


def bounds(basis_all: np.ndarray, zlo, zhi, theta) -> Dict:
    """basis_all: ncol x o x (steps+1).  Closed-form LP optimum per step."""
    basis_all = np.ascontiguousarray(basis_all, dtype=np.float64)
    ncol, o, S = basis_all.shape
    zlo = np.ascontiguousarray(zlo, dtype=np.float64)
    zhi = np.ascontiguousarray(zhi, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    lo = np.zeros((o, S))
    hi = np.zeros((o, S))
    vs, vr, ys = C.c_int(-1), C.c_int(-1), C.c_double(0.0)
    zstar = np.zeros(ncol)
    _load().ora_bounds(o, ncol, S - 1, _p(basis_all), _p(zlo), _p(zhi), _p(theta), _p(lo), _p(hi),
                       C.byref(vs), C.byref(vr), _p(zstar), C.byref(ys))
    unsafe = vs.value >= 0
    return dict(lo=lo, hi=hi, viol_step=vs.value, viol_row=vr.value,
                zstar=zstar if unsafe else None, ystar=ys.value if unsafe else None)


def checkpoints(m: int) -> List[int]:
    """Krylov dimensions at which Alg. 2 / Alg. 4 evaluate the error bound:
    k = 4, then k <- ceil(1.1 k) in IEEE double, below m."""
    import math
    out, k = [], 4
    while k < m:
        out.append(k)
        k = math.ceil(1.1 * k)
    return out


def mu_bound(system, carries_constant: bool) -> float:
    """An upper bound of the largest eigenvalue of (A + A^T)/2, the matrix the
    Krylov run of a column works on (A' = [[A, b], [0, 0]] for a column that
    carries the constant variable, else A: a generator column stays in the
    subspace where A' acts as A).

    Grid Laplacian (symmetric): the largest eigenvalue itself, the Kronecker
    sum of the 1-D Dirichlet second differences' largest eigenvalues
    -(4/h^2) sin^2(pi / (2(N+1))); with face coefficients gamma >= 0 the
    Gershgorin bound (0 for coef >= 0).  CSR: the Gershgorin bound of the symmetric
    part, max_i a_ii + (sum_{j != i} |a_ij| + |a_ji|) / 2 (+ |b_i|/2, and the
    constant row sum |b_i|/2, for A')."""
    import math
    if hasattr(system, "dims") and getattr(system, "face", None) is not None:
        # a point's Gershgorin row: -sum over its neighbours of kappa - sum
        # over its faces of gamma on the diagonal, sum of |kappa| off it
        return float(sum(2.0 * (abs(k) - k) for k in (system.coef / (h * h) for h in system.h)))
    if hasattr(system, "dims"):
        return float(sum(-system.coef * 4.0 / (h * h) * math.sin(math.pi / (2.0 * (N + 1))) ** 2
                         for N, h in zip(system.dims, system.h)))
    import scipy.sparse as sp
    n = int(system.n)
    A = sp.csr_matrix((np.asarray(system.val, dtype=np.float64), np.asarray(system.col),
                       np.asarray(system.row_ptr)), shape=(n, n))
    absA = abs(A)
    d = A.diagonal()
    off_r = np.asarray(absA.sum(axis=1)).ravel() - np.abs(d)
    off_c = np.asarray(absA.sum(axis=0)).ravel() - np.abs(d)
    g = d + 0.5 * (off_r + off_c)
    if carries_constant and system.b is not None:
        b = np.abs(np.asarray(system.b, dtype=np.float64))
        g = g + 0.5 * b
        return float(max(np.max(g), 0.5 * np.sum(b)))
    return float(np.max(g))


def lemma1(H: np.ndarray, k: int, mu: float, dt: float, steps: int) -> float:
    """The Lemma-1 bound (Sec. 4.2) for dimension k of the Krylov matrix H
    ((m+1) x m, rows beyond k unused except h_{k+1,k})."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    if k <= 0:
        return 0.0
    return float(_load().ora_lemma1(k, H.shape[1], _p(H), float(H[k, k - 1]), float(mu), float(dt), int(steps)))


def column_method(problem, col) -> str:
    """Lanczos needs a symmetric operator: the system must be symmetric and the
    column must not carry the constant variable (A' = [[A, b], [0, 0]] is not
    symmetric, but it maps {x_const = 0} into itself as A does)."""
    if problem.method in ("lanczos", "arnoldi"):
        return problem.method
    sym = bool(getattr(problem.system, "symmetric", False))
    carries = problem.system.b is not None and col.is_fixed
    return "lanczos" if (sym and not carries) else "arnoldi"


def transposed(problem) -> bool:
    """Whether the basis matrix is computed from the transpose dynamics
    (Sec. 4.1: o simulations of x' = A^T x from the rows of C, projected by
    E^T) rather than from the columns of E; "auto" takes the smaller of i
    and o, as the paper proposes."""
    mode = getattr(problem, "simulate", "forward")
    if mode == "auto":
        return problem.o < problem.i
    return mode == "transpose"


def _run_transposed(problem, sel, want_basis, eps):
    """C e^{At} E = (E^T e^{A^T t} C^T)^T: one Krylov run per output row r on
    A^T (A'^T = [[A^T, 0], [b^T, 0]] when a column carries the constant),
    from C_r^T, with the rows of E^T (the constant entry of a fixed column
    included) as the projection; basis[j][r][k] = ||C_r|| P_r[j, :] e^{H_r t_k} e_1."""
    from workloads import column_dense

    sysm = problem.system
    n = int(sysm.n)
    dims = getattr(sysm, "dims", None)
    taug = sysm.b is not None and any(c.is_fixed for c in problem.columns)
    N = n + (1 if taug else 0)
    # E'^T as CSR rows (one per column of E)
    erp, ecol, eval_ = [0], [], []
    for c in problem.columns:
        e = column_dense(c, n, dims)
        if taug:
            e = np.concatenate([e, [1.0 if c.is_fixed else 0.0]])
        nz = np.nonzero(e)[0]
        ecol.extend(nz.tolist())
        eval_.extend(e[nz].tolist())
        erp.append(len(ecol))
    erp = np.array(erp, dtype=np.int64)
    ecol = np.array(ecol, dtype=np.int64)
    eval_ = np.array(eval_, dtype=np.float64)
    sym = bool(getattr(sysm, "symmetric", False)) or dims is not None
    method = problem.method if problem.method in ("lanczos", "arnoldi") else (
        "lanczos" if (sym and not taug) else "arnoldi")
    mu = mu_bound(sysm, taug)
    crp = np.asarray(problem.C_row_ptr, dtype=np.int64)
    ccol = np.asarray(problem.C_col, dtype=np.int64)
    cval = np.asarray(problem.C_val, dtype=np.float64)
    Hs, Ps, used, beta0s, errs, checks = {}, {}, {}, {}, {}, {}
    bases = np.zeros((problem.i, problem.o, problem.steps + 1))
    for r in sel:
        c = np.zeros(N)
        np.add.at(c, ccol[crp[r]:crp[r + 1]], cval[crp[r]:crp[r + 1]])
        b0 = float(np.sqrt(np.dot(c, c)))
        beta0s[r] = b0
        if b0 == 0.0:
            Hs[r], Ps[r], used[r] = np.zeros((problem.m + 1, problem.m)), np.zeros((problem.i, problem.m)), 0
            errs[r], checks[r] = 0.0, []
            continue
        H, P, u = krylov(sysm, c / b0, problem.m, erp, ecol, eval_, method=method, aug=taug, trans=True)
        checks[r] = []
        if eps > 0.0:
            for k in checkpoints(problem.m):
                if k >= u:
                    break
                ek = lemma1(H, k, mu, problem.dt, problem.steps)
                checks[r].append((k, ek))
                if ek < eps:
                    u = k
                    break
        errs[r] = lemma1(H, u, mu, problem.dt, problem.steps)
        Hs[r], Ps[r], used[r] = H, P, u
        if want_basis:
            bases[:, r, :] = basis(H, P, u, b0, problem.dt, problem.steps)
    out = dict(H=Hs, P=Ps, used=used, beta0=beta0s, err=errs, checks=checks, transposed=True,
               basis={j: bases[j] for j in range(problem.i)})
    if want_basis and len(sel) == problem.o:
        zlo = [c.zlo for c in problem.columns]
        zhi = [c.zhi for c in problem.columns]
        out.update(bounds(bases, zlo, zhi, problem.theta))
    return out


def run(problem, *, columns: Optional[List[int]] = None, want_basis: bool = True) -> Dict:
    """The whole path for one problem.  `columns` restricts the Krylov runs to
    a subset of the initial-space columns (for sampled checks on large cases;
    of the output rows when the transpose dynamics run); bounds are then only
    computed when every run was made."""
    from workloads import column_dense

    if transposed(problem):
        eps_t = float(getattr(problem, "err_target", 0.0) or 0.0)
        sel_t = list(range(problem.o)) if columns is None else list(columns)
        return _run_transposed(problem, sel_t, want_basis, eps_t)

    sysm = problem.system
    n = int(sysm.n)
    dims = getattr(sysm, "dims", None)
    aug = sysm.b is not None
    sel = list(range(problem.i)) if columns is None else list(columns)
    Hs, Ps, used, beta0s, bases, errs, checks = {}, {}, {}, {}, {}, {}, {}
    eps = float(getattr(problem, "err_target", 0.0) or 0.0)
    for j in sel:
        col = problem.columns[j]
        e = column_dense(col, n, dims)
        if aug:
            e = np.concatenate([e, [1.0 if col.is_fixed else 0.0]])
        b0 = float(np.sqrt(np.dot(e, e)))
        beta0s[j] = b0
        if b0 == 0.0:
            Hs[j] = np.zeros((problem.m + 1, problem.m))
            Ps[j] = np.zeros((problem.o, problem.m))
            used[j] = 0
            bases[j] = np.zeros((problem.o, problem.steps + 1))
            errs[j], checks[j] = 0.0, []
            continue
        H, P, u = krylov(sysm, e / b0, problem.m, problem.C_row_ptr, problem.C_col, problem.C_val,
                         method=column_method(problem, col), aug=aug)
        # Alg. 2 / Alg. 4: the first checkpoint below the dimension reached
        # whose bound is under the target ends the iteration there
        mu = mu_bound(sysm, aug and bool(col.is_fixed))
        checks[j] = []
        if eps > 0.0:
            for k in checkpoints(problem.m):
                if k >= u:
                    break
                ek = lemma1(H, k, mu, problem.dt, problem.steps)
                checks[j].append((k, ek))
                if ek < eps:
                    u = k
                    break
        errs[j] = lemma1(H, u, mu, problem.dt, problem.steps)
        Hs[j], Ps[j], used[j] = H, P, u
        if want_basis:
            bases[j] = basis(H, P, u, b0, problem.dt, problem.steps)
    out = dict(H=Hs, P=Ps, used=used, beta0=beta0s, basis=bases, err=errs, checks=checks)
    if want_basis and len(sel) == problem.i:
        ball = np.stack([bases[j] for j in range(problem.i)])
        zlo = [c.zlo for c in problem.columns]
        zhi = [c.zhi for c in problem.columns]
        out.update(bounds(ball, zlo, zhi, problem.theta))
    return out
