"""Python binding of libkv (include/kv.h): argument marshalling only.

Every step of the verification path runs in the CUDA library; this module
packs Python/numpy arguments into the C structures, calls the entry point of
the same name and unpacks the results.  PyTorch, when used, only provides the
device pool and the stream.  There is no fallback: if libkv.so is missing the
first call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# KV_LIBRARY: another build of the library (the debug build of build.py)
LIB_PATH = os.environ.get("KV_LIBRARY") or os.path.join(_HERE, "_build", "libkv.so")

KV_OK, KV_EINVAL, KV_ENOMEM, KV_ECUDA, KV_ETIMEOUT, KV_EBUSY, KV_ENOTREADY = range(7)
KV_FP64, KV_FP32 = 0, 1
KV_AUTO, KV_LANCZOS, KV_ARNOLDI = 0, 1, 2
KV_COL_BOX, KV_COL_SPARSE, KV_COL_DENSE = 0, 1, 2
KV_EXPM_PER_STEP, KV_EXPM_PROPAGATE = 0, 1
KV_MAX_M = 256
KV_MAX_M_LANCZOS = 4096
KV_FLAG_TWO_PASS = 1

KV_PREC_AUTO = 2
_PREC = {"fp64": KV_FP64, "fp32": KV_FP32, "auto": KV_PREC_AUTO}
_METH = {"auto": KV_AUTO, "lanczos": KV_LANCZOS, "arnoldi": KV_ARNOLDI}
_EXPM = {"per_step": KV_EXPM_PER_STEP, "propagate": KV_EXPM_PROPAGATE}
KV_SIM_FORWARD, KV_SIM_TRANSPOSE, KV_SIM_AUTO = 0, 1, 2
_SIM = {"forward": KV_SIM_FORWARD, "transpose": KV_SIM_TRANSPOSE, "auto": KV_SIM_AUTO}


def runs_of(problem):
    """(runs, transposed): the Krylov runs a problem makes -- one per column
    of E, or one per row of C with the transpose dynamics (the library's
    rule: "auto" transposes when o < i)."""
    mode = getattr(problem, "simulate", "forward")
    tr = mode == "transpose" or (mode == "auto" and problem.o < problem.i)
    return (problem.o if tr else problem.i), tr


class KvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"kv error {code}: {msg}")
        self.code = code


class kv_column(C.Structure):
    _fields_ = [("kind", C.c_int32), ("is_fixed", C.c_int32), ("zlo", C.c_double), ("zhi", C.c_double),
                ("box_lo", C.c_int64 * 3), ("box_hi", C.c_int64 * 3), ("value", C.c_double),
                ("nnz", C.c_int64), ("idx", C.c_void_p), ("val", C.c_void_p), ("dense", C.c_void_p)]


class kv_problem_desc(C.Structure):
    _fields_ = [("i", C.c_int32), ("cols", C.POINTER(kv_column)), ("o", C.c_int32),
                ("c_row_ptr", C.c_void_p), ("c_col", C.c_void_p), ("c_val", C.c_void_p),
                ("theta", C.c_void_p), ("dt", C.c_double), ("steps", C.c_int32),
                ("krylov_m", C.c_int32), ("method", C.c_int32), ("expm_mode", C.c_int32),
                ("batched", C.c_int32), ("flags", C.c_int32), ("err_target", C.c_double),
                ("simulate", C.c_int32)]


class kv_result(C.Structure):
    _fields_ = [("lo", C.c_void_p), ("hi", C.c_void_p), ("basis", C.c_void_p), ("H", C.c_void_p),
                ("P", C.c_void_p), ("beta0", C.c_void_p), ("m_used", C.c_void_p), ("z_star", C.c_void_p),
                ("first_violation_step", C.c_int32), ("violation_row", C.c_int32), ("y_star", C.c_double),
                ("err_bound", C.c_void_p)]


class kv_polytope(C.Structure):
    _fields_ = [("rows", C.c_int32), ("a", C.c_void_p), ("rhs", C.c_void_p)]


class kv_lp_result(C.Structure):
    _fields_ = [("margin", C.c_void_p), ("status", C.c_void_p), ("z", C.c_void_p),
                ("first_violation_step", C.c_int32), ("z_star", C.c_void_p), ("y_star", C.c_void_p)]


KV_LP_OPTIMAL, KV_LP_FAILED, KV_LP_EMPTY, KV_LP_ITER = 0, 1, 2, 3

EXPORTED = ["kv_version", "kv_last_error", "kv_create", "kv_destroy", "kv_pool_stats", "kv_system_stencil",
            "kv_system_grid",
            "kv_system_csr", "kv_sys_destroy", "kv_problem", "kv_prob_destroy", "kv_problem_bytes",
            "kv_enqueue", "kv_fetch", "kv_run", "kv_profile_enable", "kv_profile_read", "kv_launch_count",
            "kv_problem_runs", "kv_diag_bounded_wait", "kv_check_polytope", "kv_diag_fp64_rate",
            "kv_problem_precision"]

_lib = None
_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load libkv.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libkv.so not found at {p}: run __graft_entry__.build() first "
                               "(the CUDA library is required; there is no CPU fallback)")
        lib = C.CDLL(p)
        V = C.c_void_p
        I = C.c_int
        lib.kv_version.restype = C.c_char_p
        lib.kv_last_error.restype = C.c_char_p
        lib.kv_create.argtypes = [C.POINTER(V), I, V, C.c_size_t, V]
        lib.kv_destroy.argtypes = [V]
        lib.kv_pool_stats.argtypes = [V, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        lib.kv_system_stencil.argtypes = [V, C.POINTER(V), I, C.POINTER(C.c_int64), C.c_double,
                                          C.POINTER(C.c_double), V]
        lib.kv_system_grid.argtypes = [V, C.POINTER(V), I, C.POINTER(C.c_int64), C.c_double,
                                       C.POINTER(C.c_double), V, V]
        lib.kv_system_csr.argtypes = [V, C.POINTER(V), C.c_int64, V, V, V, V, I, I, I]
        lib.kv_diag_fp64_rate.argtypes = [I, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.kv_sys_destroy.argtypes = [V]
        lib.kv_problem.argtypes = [V, C.POINTER(V), V, C.POINTER(kv_problem_desc), I]
        lib.kv_prob_destroy.argtypes = [V]
        lib.kv_problem_bytes.argtypes = [V, C.POINTER(kv_problem_desc), I, C.POINTER(C.c_size_t)]
        lib.kv_enqueue.argtypes = [V]
        lib.kv_fetch.argtypes = [V, C.POINTER(kv_result)]
        lib.kv_run.argtypes = [V, C.POINTER(kv_result)]
        lib.kv_profile_enable.argtypes = [V, I]
        lib.kv_profile_read.argtypes = [V, C.c_char_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        lib.kv_launch_count.argtypes = [V, C.POINTER(C.c_int64)]
        lib.kv_problem_runs.argtypes = [V, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        lib.kv_diag_bounded_wait.argtypes = [I, C.c_int64]
        lib.kv_check_polytope.argtypes = [V, C.POINTER(kv_polytope), C.POINTER(kv_polytope), C.c_double,
                                          C.POINTER(kv_lp_result)]
        lib.kv_grid_lanczos_noalloc.argtypes = [I, V, I, C.POINTER(C.c_int64), C.c_double, C.POINTER(C.c_double),
                                                C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_double, C.c_int32,
                                                V, V, V, C.c_int32, V, V, V, V]
        lib.kv_grid_lanczos_noalloc.restype = C.c_int
        for name in EXPORTED:
            f = getattr(lib, name)
            if f.restype is None and name not in ("kv_version", "kv_last_error"):
                f.restype = C.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != KV_OK:
        raise KvError(rc, last_error())


def version() -> str:
    return load().kv_version().decode()


def last_error() -> str:
    return load().kv_last_error().decode()


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
class Context:
    """kv_create / kv_destroy.  pool: None (library allocates pool_bytes once)
    or a torch CUDA tensor used as the pool; stream: None or a torch stream."""

    def __init__(self, pool_bytes: int, device: int = 0, pool=None, stream=None):
        self._lib = load()
        self._pool = pool
        h = C.c_void_p()
        pool_ptr = None if pool is None else C.c_void_p(pool.data_ptr())
        if pool is not None:
            pool_bytes = pool.numel() * pool.element_size()
        stream_ptr = None if stream is None else C.c_void_p(stream.cuda_stream)
        _check(self._lib.kv_create(C.byref(h), device, pool_ptr, pool_bytes, stream_ptr))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.kv_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pool_stats(self):
        a, b = C.c_size_t(), C.c_size_t()
        _check(self._lib.kv_pool_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def launch_count(self) -> int:
        n = C.c_int64()
        _check(self._lib.kv_launch_count(self.h, C.byref(n)))
        return n.value

    def profile_enable(self, on: bool = True):
        _check(self._lib.kv_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, name: str):
        n, t = C.c_int64(), C.c_double()
        _check(self._lib.kv_profile_read(self.h, name.encode(), C.byref(n), C.byref(t)))
        return n.value, t.value


class System:
    """kv_system_stencil (kv_system_grid when the grid has face coefficients) /
    kv_system_csr / kv_sys_destroy for a workloads system."""

    def __init__(self, ctx: Context, system, precision: str = "fp64"):
        self.ctx = ctx
        lib = ctx._lib
        h = C.c_void_p()
        b = getattr(system, "b", None)
        bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
        if hasattr(system, "dims"):
            nd = len(system.dims)
            dims = (C.c_int64 * 3)(*[int(system.dims[a]) if a < nd else 1 for a in range(3)])
            hh = (C.c_double * 3)(*[float(system.h[a]) if a < nd else 1.0 for a in range(3)])
            face = getattr(system, "face", None)
            if face is None:
                _check(lib.kv_system_stencil(ctx.h, C.byref(h), nd, dims, float(system.coef), hh, _ptr(bb)))
            else:
                ff = np.ascontiguousarray(face, dtype=np.float64)
                if ff.shape != (2 * nd,):
                    raise ValueError(f"face must hold {2 * nd} coefficients")
                _check(lib.kv_system_grid(ctx.h, C.byref(h), nd, dims, float(system.coef), hh, _ptr(ff), _ptr(bb)))
        else:
            rp = np.ascontiguousarray(system.row_ptr, dtype=np.int64)
            col = np.ascontiguousarray(system.col, dtype=np.int32)
            val = np.ascontiguousarray(system.val, dtype=np.float64)
            _check(lib.kv_system_csr(ctx.h, C.byref(h), int(system.n), _ptr(rp), _ptr(col), _ptr(val), _ptr(bb),
                                     1 if system.symmetric else 0,
                                     KV_FP64 if precision == "auto" else _PREC[precision], 0))
        self.h = h
        self.n = int(system.n)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.ctx._lib.kv_sys_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(problem, expm_mode: str, batched: bool, keep: list, flags: int = 0) -> kv_problem_desc:
    cols = (kv_column * problem.i)()
    for j, c in enumerate(problem.columns):
        cc = cols[j]
        cc.is_fixed = 1 if c.is_fixed else 0
        cc.zlo, cc.zhi = float(c.zlo), float(c.zhi)
        if c.kind == "box":
            cc.kind = KV_COL_BOX
            for a in range(3):
                cc.box_lo[a] = int(c.box_lo[a]) if a < len(c.box_lo) else 0
                cc.box_hi[a] = int(c.box_hi[a]) if a < len(c.box_hi) else 1
            cc.value = float(c.value)
        elif c.kind == "sparse":
            cc.kind = KV_COL_SPARSE
            ix = np.ascontiguousarray(c.idx, dtype=np.int64)
            vv = np.ascontiguousarray(c.val, dtype=np.float64)
            keep += [ix, vv]
            cc.nnz = len(ix)
            cc.idx, cc.val = _ptr(ix), _ptr(vv)
        elif c.kind == "dense":
            cc.kind = KV_COL_DENSE
            dd = np.ascontiguousarray(c.dense, dtype=np.float64)
            keep.append(dd)
            cc.dense = _ptr(dd)
        else:
            raise ValueError(c.kind)
    rp = np.ascontiguousarray(problem.C_row_ptr, dtype=np.int64)
    cc_ = np.ascontiguousarray(problem.C_col, dtype=np.int64)
    cv = np.ascontiguousarray(problem.C_val, dtype=np.float64)
    th = np.ascontiguousarray(problem.theta, dtype=np.float64)
    keep += [cols, rp, cc_, cv, th]
    d = kv_problem_desc()
    d.i = problem.i
    d.cols = C.cast(cols, C.POINTER(kv_column))
    d.o = problem.o
    d.c_row_ptr, d.c_col, d.c_val, d.theta = _ptr(rp), _ptr(cc_), _ptr(cv), _ptr(th)
    d.dt = float(problem.dt)
    d.steps = int(problem.steps)
    d.krylov_m = int(problem.m)
    d.method = _METH[problem.method]
    d.expm_mode = _EXPM[expm_mode]
    d.batched = 1 if batched else 0
    d.flags = int(flags)
    d.err_target = float(getattr(problem, "err_target", 0.0) or 0.0)
    d.simulate = _SIM[getattr(problem, "simulate", "forward")]
    return d


class ProblemHandle:
    """kv_problem / kv_enqueue / kv_fetch / kv_run / kv_prob_destroy."""

    def __init__(self, ctx: Context, sysh: System, problem, *, expm_mode: str = "per_step",
                 batched: bool = False, flags: int = 0):
        self.ctx = ctx
        self.sysh = sysh
        self.problem = problem
        self._keep: list = []
        self.desc = _desc(problem, expm_mode, batched, self._keep, flags)
        h = C.c_void_p()
        _check(ctx._lib.kv_problem(ctx.h, C.byref(h), sysh.h, C.byref(self.desc), _PREC[problem.precision]))
        self.h = h
        runs, tr = C.c_int32(), C.c_int32()
        _check(ctx._lib.kv_problem_runs(h, C.byref(runs), C.byref(tr)))
        self.runs, self.transposed = int(runs.value), bool(tr.value)
        prec = C.c_int32()
        _check(ctx._lib.kv_problem_precision(h, C.byref(prec)))
        self.precision = "fp64" if prec.value == KV_FP64 else "fp32"

    def enqueue(self):
        _check(self.ctx._lib.kv_enqueue(self.h))

    def fetch(self, full: bool = True) -> Dict:
        p = self.problem
        S = p.steps + 1
        out = dict(lo=np.zeros((p.o, S)), hi=np.zeros((p.o, S)))
        R = self.runs                        # per-run arrays (o runs with the transpose dynamics)
        prow = p.i if self.transposed else p.o  # rows of each run's P
        if full:
            out.update(basis=np.zeros((p.i, p.o, S)), H=np.zeros((R, p.m + 1, p.m)),
                       P=np.zeros((R, prow, p.m)), beta0=np.zeros(R), m_used=np.zeros(R, dtype=np.int32))
        out["zstar"] = np.zeros(p.i)
        out["err_bound"] = np.zeros(R)
        out["transposed"] = self.transposed
        r = kv_result()
        r.lo, r.hi = _ptr(out["lo"]), _ptr(out["hi"])
        r.err_bound = _ptr(out["err_bound"])
        if full:
            r.basis, r.H, r.P = _ptr(out["basis"]), _ptr(out["H"]), _ptr(out["P"])
            r.beta0, r.m_used = _ptr(out["beta0"]), _ptr(out["m_used"])
        r.z_star = _ptr(out["zstar"])
        _check(self.ctx._lib.kv_fetch(self.h, C.byref(r)))
        out["viol_step"] = int(r.first_violation_step)
        out["viol_row"] = int(r.violation_row)
        if out["viol_step"] < 0:
            out["zstar"] = None
            out["ystar"] = None
        else:
            out["ystar"] = float(r.y_star)
        return out

    def run(self, full: bool = True) -> Dict:
        self.enqueue()
        return self.fetch(full)

    def check_polytope(self, U, v, Iz=None, iota=None, tol: float = 0.0) -> Dict:
        """kv_check_polytope: the per-step LP margins t*_k for the unsafe set
        U y <= v (rows over the o outputs) and the initial set of the columns'
        boxes with I_z z <= iota; the first step with t*_k <= tol, its z*, y*."""
        p = self.problem
        S = p.steps + 1
        U = np.ascontiguousarray(np.atleast_2d(np.asarray(U, dtype=np.float64)))
        v = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
        if U.shape != (len(v), p.o):
            raise ValueError(f"unsafe rows must be {len(v)} x {p.o}")
        un = kv_polytope(len(v), _ptr(U), _ptr(v))
        ini = None
        if Iz is not None and len(Iz):
            Iz = np.ascontiguousarray(np.atleast_2d(np.asarray(Iz, dtype=np.float64)))
            iota = np.ascontiguousarray(np.asarray(iota, dtype=np.float64).reshape(-1))
            if Iz.shape != (len(iota), p.i):
                raise ValueError(f"initial rows must be {len(iota)} x {p.i}")
            ini = kv_polytope(len(iota), _ptr(Iz), _ptr(iota))
        out = dict(margin=np.zeros(S), status=np.zeros(S, dtype=np.int32), z=np.zeros((S, p.i)),
                   z_star=np.zeros(p.i), y_star=np.zeros(p.o))
        r = kv_lp_result()
        r.margin, r.status, r.z = _ptr(out["margin"]), _ptr(out["status"]), _ptr(out["z"])
        r.z_star, r.y_star = _ptr(out["z_star"]), _ptr(out["y_star"])
        _check(self.ctx._lib.kv_check_polytope(self.h, C.byref(un), C.byref(ini) if ini is not None else None,
                                               float(tol), C.byref(r)))
        out["viol_step"] = int(r.first_violation_step)
        if out["viol_step"] < 0:
            out["z_star"] = out["y_star"] = None
        return out

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.ctx._lib.kv_prob_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """kv_graph_create / kv_graph_launch / kv_graph_destroy over ProblemHandles
    created on the same context."""

    def __init__(self, ctx: Context, handles):
        self.ctx = ctx
        lib = ctx._lib
        if not getattr(lib, "_graph_ready", False):
            lib.kv_graph_create.argtypes = [C.c_void_p, C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]
            lib.kv_graph_launch.argtypes = [C.c_void_p]
            lib.kv_graph_destroy.argtypes = [C.c_void_p]
            for f in (lib.kv_graph_create, lib.kv_graph_launch, lib.kv_graph_destroy):
                f.restype = C.c_int
            lib._graph_ready = True
        self.handles = list(handles)
        arr = (C.c_void_p * len(self.handles))(*[h.h.value for h in self.handles])
        g = C.c_void_p()
        _check(lib.kv_graph_create(ctx.h, arr, len(self.handles), C.byref(g)))
        self.h = g

    def launch(self):
        _check(self.ctx._lib.kv_graph_launch(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.ctx._lib.kv_graph_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class kv_query(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ndim", C.c_int32), ("dims", C.c_int64 * 3), ("coef", C.c_double),
                ("h", C.c_double * 3), ("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("symmetric", C.c_int32), ("b", C.c_void_p), ("desc", kv_problem_desc),
                ("precision", C.c_int32), ("face", C.c_void_p)]


def _load_server(lib):
    if getattr(lib, "_server_ready", False):
        return
    V = C.c_void_p
    lib.kv_server_create.argtypes = [V, C.POINTER(V), C.c_int32]
    lib.kv_server_destroy.argtypes = [V]
    lib.kv_submit.argtypes = [V, C.POINTER(kv_query), C.POINTER(C.c_uint64)]
    lib.kv_poll.argtypes = [V, C.c_uint64, C.POINTER(kv_result), C.POINTER(C.c_double)]
    lib.kv_server_stats.argtypes = [V, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    lib.kv_server_system_stats.argtypes = [V] + [C.POINTER(C.c_int64)] * 4
    for f in (lib.kv_server_create, lib.kv_server_destroy, lib.kv_submit, lib.kv_poll, lib.kv_server_stats,
              lib.kv_server_system_stats):
        f.restype = C.c_int
    lib._server_ready = True


class Server:
    """kv_server_create / kv_submit / kv_poll / kv_server_stats / kv_server_destroy.
    The context belongs to the server's worker until close()."""

    def __init__(self, ctx: Context, slots: int = 8):
        self.ctx = ctx
        self._lib = ctx._lib
        _load_server(self._lib)
        h = C.c_void_p()
        _check(self._lib.kv_server_create(ctx.h, C.byref(h), int(slots)))
        self.h = h
        self._keep: Dict[int, tuple] = {}
        # converted host arrays per system object while a query names it, so
        # that queries on one CSR system pass the same pointers and share its
        # device copy: id -> [system, arrays, queries]
        self._arrays: Dict[int, list] = {}

    def _system_arrays(self, s) -> tuple:
        ent = self._arrays.get(id(s))
        if ent is None:
            b = getattr(s, "b", None)
            bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
            if hasattr(s, "dims"):
                face = getattr(s, "face", None)
                ff = None if face is None else np.ascontiguousarray(face, dtype=np.float64)
                if ff is not None and ff.shape != (2 * len(s.dims),):
                    raise ValueError(f"face must hold {2 * len(s.dims)} coefficients")
                arrs = (bb, ff)
            else:
                arrs = (bb, np.ascontiguousarray(s.row_ptr, dtype=np.int64),
                        np.ascontiguousarray(s.col, dtype=np.int32), np.ascontiguousarray(s.val, dtype=np.float64))
            ent = self._arrays[id(s)] = [s, arrs, 0]
        ent[2] += 1
        return ent[1]

    def _release_arrays(self, s):
        ent = self._arrays.get(id(s))
        if ent is not None:
            ent[2] -= 1
            if ent[2] == 0:
                del self._arrays[id(s)]

    def submit(self, problem, *, expm_mode: str = "propagate", flags: int = 0) -> int:
        s = problem.system
        arrs = self._system_arrays(s)
        try:
            q, keep, t = self._submit(problem, s, arrs, expm_mode, flags)
        except Exception:
            self._release_arrays(s)
            raise
        self._keep[t] = (q, keep, problem)
        return t

    def _submit(self, problem, s, arrs, expm_mode, flags):
        keep: list = [a for a in arrs if a is not None]
        q = kv_query()
        if arrs[0] is not None:
            q.b = _ptr(arrs[0])
        if hasattr(s, "dims"):
            q.kind = 0
            q.face = _ptr(arrs[1])
            q.ndim = len(s.dims)
            for a in range(3):
                q.dims[a] = int(s.dims[a]) if a < q.ndim else 1
                q.h[a] = float(s.h[a]) if a < q.ndim else 1.0
            q.coef = float(s.coef)
        else:
            q.kind = 1
            rp, col, val = arrs[1:]
            q.n = int(s.n)
            q.row_ptr, q.col, q.val = _ptr(rp), _ptr(col), _ptr(val)
            q.symmetric = 1 if s.symmetric else 0
        q.desc = _desc(problem, expm_mode, False, keep, flags)
        q.precision = _PREC[problem.precision]
        t = C.c_uint64()
        _check(self._lib.kv_submit(self.h, C.byref(q), C.byref(t)))
        return q, keep, t.value

    def poll(self, ticket: int) -> Optional[Dict]:
        """None while queued or running; the results once finished (raises
        KvError if the query failed)."""
        q, keep, p = self._keep[ticket]
        S = p.steps + 1
        R, _ = runs_of(p)
        out = dict(lo=np.zeros((p.o, S)), hi=np.zeros((p.o, S)), beta0=np.zeros(R),
                   m_used=np.zeros(R, dtype=np.int32), zstar=np.zeros(p.i), err_bound=np.zeros(R))
        r = kv_result()
        r.lo, r.hi, r.beta0, r.m_used, r.z_star = (_ptr(out["lo"]), _ptr(out["hi"]), _ptr(out["beta0"]),
                                                   _ptr(out["m_used"]), _ptr(out["zstar"]))
        r.err_bound = _ptr(out["err_bound"])
        lat = C.c_double()
        rc = self._lib.kv_poll(self.h, ticket, C.byref(r), C.byref(lat))
        if rc == KV_ENOTREADY:
            return None
        del self._keep[ticket]
        self._release_arrays(p.system)
        _check(rc)
        out["viol_step"] = int(r.first_violation_step)
        out["viol_row"] = int(r.violation_row)
        out["ystar"] = float(r.y_star) if out["viol_step"] >= 0 else None
        if out["viol_step"] < 0:
            out["zstar"] = None
        out["latency_ms"] = float(lat.value)
        return out

    def stats(self) -> Dict:
        a, c, pnd, mw = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        mr = C.c_int32()
        _check(self._lib.kv_server_stats(self.h, C.byref(a), C.byref(c), C.byref(pnd), C.byref(mr), C.byref(mw)))
        b, u, r, n = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._lib.kv_server_system_stats(self.h, C.byref(b), C.byref(u), C.byref(r), C.byref(n)))
        return dict(admitted=a.value, completed=c.value, pending=pnd.value, max_running=mr.value,
                    memory_waits=mw.value, systems_built=b.value, systems_reused=u.value,
                    systems_released=r.value, systems_resident=n.value)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.kv_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


KV_NOALLOC_MAX_N = 262144


def debug_set_c_col(ph: "ProblemHandle", e: int, value: int) -> None:
    """kv_debug_set_c_col (debug build only): overwrite entry e of the
    problem's device copy of C's column indices."""
    lib = load()
    if not hasattr(lib, "kv_debug_set_c_col"):
        raise RuntimeError("kv_debug_set_c_col exists in the debug build only (build(debug=True), KV_LIBRARY)")
    f = lib.kv_debug_set_c_col
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
    f.restype = C.c_int
    _check(f(ph.h, int(e), int(value)))


def diag_fp64_rate(device: int = 0):
    """kv_diag_fp64_rate: (FP64 FMA/s, FP64 add/s) measured on the device."""
    lib = load()
    f, a = C.c_double(), C.c_double()
    _check(lib.kv_diag_fp64_rate(device, C.byref(f), C.byref(a)))
    return f.value, a.value


def grid_lanczos_noalloc(device: int, stream, ndim: int, dims, coef: float, h, box_lo, box_hi, value: float,
                         o: int, c_row_ptr, c_col, c_val, krylov_m: int, H, P, beta0, m_used) -> None:
    """kv_grid_lanczos_noalloc: every array argument is a device pointer (an
    int) owned by the caller; stream is a cudaStream_t as an int, or None.
    The library allocates nothing for this call (see include/kv.h)."""
    lib = load()
    d3 = (C.c_int64 * 3)(*[int(dims[a]) if a < len(dims) else 1 for a in range(3)])
    h3 = (C.c_double * 3)(*[float(h[a]) if a < len(h) else 1.0 for a in range(3)])
    lo3 = (C.c_int64 * 3)(*[int(box_lo[a]) if a < len(box_lo) else 0 for a in range(3)])
    hi3 = (C.c_int64 * 3)(*[int(box_hi[a]) if a < len(box_hi) else 1 for a in range(3)])
    _check(lib.kv_grid_lanczos_noalloc(device, stream, ndim, d3, float(coef), h3, lo3, hi3, float(value), o,
                                       c_row_ptr, c_col, c_val, krylov_m, H, P, beta0, m_used))


def problem_bytes(sysh: System, problem, *, expm_mode: str = "per_step", batched: bool = False,
                  flags: int = 0) -> int:
    keep: list = []
    d = _desc(problem, expm_mode, batched, keep, flags)
    n = C.c_size_t()
    _check(sysh.ctx._lib.kv_problem_bytes(sysh.h, C.byref(d), _PREC[problem.precision], C.byref(n)))
    return n.value


def solve(problem, ctx: Optional[Context] = None, *, pool_bytes: int = 1 << 30, expm_mode: str = "per_step",
          batched: bool = False, flags: int = 0) -> Dict:
    """Convenience: system + problem + run on a (new) context."""
    own = ctx is None
    if own:
        ctx = Context(pool_bytes)
    sysh = System(ctx, problem.system, problem.precision)
    ph = ProblemHandle(ctx, sysh, problem, expm_mode=expm_mode, batched=batched, flags=flags)
    try:
        return ph.run()
    finally:
        ph.close()
        sysh.close()
        if own:
            ctx.close()


def diag_bounded_wait(polls: int, device: int = 0) -> int:
    """kv_diag_bounded_wait: the status code (KV_ETIMEOUT when the bounded
    wait expired, as it must)."""
    return int(load().kv_diag_bounded_wait(int(device), int(polls)))
