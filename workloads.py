"""Seeded synthetic inputs for the projected-Krylov verification path.

This module only *describes* problems: grids, sparse matrices, initial-set
columns, output rows and thresholds, drawn from fixed seeds.  It holds none of
the method's arithmetic (no Krylov step, no exponential, no bound), so both the
CPU oracle and the CUDA path can be fed from it without sharing any of the
computation they are compared on.

Workload shapes follow the paper's benchmarks:
  * 2D / 3D heat diffusion on a uniform grid with a Dirichlet-0 boundary, a
    heated block as a one-generator initial set and the temperature at the
    centre as output (Sec. 5.3, "Symmetric 3D Heat Diffusion");
  * a random sparse nonsymmetric system with a forcing term b, a box initial
    set over a few variables and a couple of +-1 output rows, standing in for
    the circuit benchmark of Sec. 5.1 (its matrix is not available);
  * the timed harmonic oscillator worked example of Sec. 2.2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


# --------------------------------------------------------------------------
# descriptions
# --------------------------------------------------------------------------
@dataclass
class GridSystem:
    """dx/dt = coef * Laplacian_h(x) (+ b), Dirichlet-0 outside the grid
    unless `face` gives a coefficient per face of the grid box.

    dims are (nx, ny) or (nx, ny, nz); x varies fastest in the flat index
    idx = (z*ny + y)*nx + x.  h holds the grid spacing per axis.  face:
    None, or 2*ndim values gamma_f >= 0 (x low, x high, y low, y high, z
    low, z high): a point on face f gets -gamma_f x_p in place of the coupling
    coef/h_a^2 (x_q - x_p) to its missing neighbour (coef/h_a^2 is the
    Dirichlet-0 ghost, 0 an insulated face).
    """
    dims: Tuple[int, ...]
    coef: float
    h: Tuple[float, ...]
    b: Optional[np.ndarray] = None
    face: Optional[Tuple[float, ...]] = None

    @property
    def ndim(self) -> int:
        return len(self.dims)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims, dtype=np.int64))

    symmetric = True  # the Dirichlet Laplacian is symmetric


@dataclass
class CsrSystem:
    """dx/dt = A x (+ b) with A in CSR form (row_ptr int64, col int32, val f64)."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    b: Optional[np.ndarray] = None
    symmetric: bool = False


@dataclass
class Column:
    """One column E_j of the initial-space matrix, x0 = sum_j E_j z_j.

    kind = "box":    E_j = value on the grid cells lo <= idx < hi (per axis)
    kind = "sparse": E_j[idx] = val
    kind = "dense":  E_j = dense (length n)
    is_fixed: z_j is pinned to 1 and the column carries the constant-1
    variable used to fold b into the dynamics (Sec. 2.1).
    """
    kind: str
    zlo: float
    zhi: float
    is_fixed: bool = False
    box_lo: Tuple[int, ...] = ()
    box_hi: Tuple[int, ...] = ()
    value: float = 1.0
    idx: Optional[np.ndarray] = None
    val: Optional[np.ndarray] = None
    dense: Optional[np.ndarray] = None


@dataclass
class Problem:
    system: object
    columns: List[Column]
    C_row_ptr: np.ndarray
    C_col: np.ndarray
    C_val: np.ndarray
    theta: np.ndarray          # per output row; +inf = no check
    dt: float
    steps: int
    m: int                     # Krylov dimension (the paper's k)
    method: str = "auto"       # auto | lanczos | arnoldi
    precision: str = "fp64"    # fp64 | fp32
    name: str = ""
    err_target: float = 0.0    # > 0: a-posteriori error control with m as the maximum dimension
    simulate: str = "forward"  # forward | transpose | auto (the smaller of i and o runs)

    @property
    def o(self) -> int:
        return len(self.C_row_ptr) - 1

    @property
    def i(self) -> int:
        return len(self.columns)


def _c_rows(rows: Sequence[Tuple[Sequence[int], Sequence[float]]]):
    rp = [0]
    cols: List[int] = []
    vals: List[float] = []
    for idx, val in rows:
        cols.extend(int(c) for c in idx)
        vals.extend(float(v) for v in val)
        rp.append(len(cols))
    return (np.asarray(rp, dtype=np.int64), np.asarray(cols, dtype=np.int64),
            np.asarray(vals, dtype=np.float64))


def grid_index(dims: Sequence[int], cell: Sequence[int]) -> int:
    idx = 0
    for ax in reversed(range(len(dims))):
        idx = idx * int(dims[ax]) + int(cell[ax])
    return idx


# --------------------------------------------------------------------------
# heat diffusion (Sec. 5.3 shapes; Dirichlet-0 boundary)
# --------------------------------------------------------------------------
def heat(dims: Sequence[int], *, coef: float = 0.01, block: Sequence[int],
         output: str = "centre", theta: float = math.inf, dt: float,
         steps: int, m: int, zlo: float = 0.9, zhi: float = 1.1,
         precision: str = "fp64", method: str = "auto", name: str = "") -> Problem:
    """Heat equation on a grid with spacing h = 1/(N+1) per axis.

    Initial set: the corner block [0, block) per axis at temperature
    u in [zlo, zhi] (one generator, one Krylov run); everything else 0.
    output = "centre": the cell N//2 on every axis;
    output = "centre8": the mean of the 2^ndim cells {N//2-1, N//2}^ndim;
    output = "edge": the cell just past the block's far corner (block[a] on
    every axis), one stencil application per axis from the block, so the
    Krylov space reaches it after ndim steps (the centre lies beyond the
    reach of m stencil applications on large grids, where the projected
    output is exactly 0).
    """
    dims = tuple(int(d) for d in dims)
    h = tuple(1.0 / (d + 1) for d in dims)
    sysm = GridSystem(dims=dims, coef=coef, h=h)
    col = Column(kind="box", zlo=zlo, zhi=zhi, box_lo=tuple(0 for _ in dims),
                 box_hi=tuple(int(b) for b in block), value=1.0)
    if output == "centre":
        cells = [tuple(d // 2 for d in dims)]
    elif output == "centre8":
        import itertools
        cells = list(itertools.product(*[(d // 2 - 1, d // 2) for d in dims]))
    elif output == "edge":
        cells = [tuple(min(int(b), d - 1) for b, d in zip(block, dims))]
    else:
        raise ValueError(output)
    w = 1.0 / len(cells)
    rp, cc, cv = _c_rows([([grid_index(dims, c) for c in cells], [w] * len(cells))])
    return Problem(system=sysm, columns=[col], C_row_ptr=rp, C_col=cc, C_val=cv,
                   theta=np.array([theta]), dt=dt, steps=steps, m=m,
                   method=method, precision=precision, name=name)


def heat2d_20(**kw) -> Problem:
    """20x20 grid, 5x5 heated corner block, output at cell (10,10),
    unsafe y >= 0.05, dt 0.1, 500 steps, Lanczos m = 30."""
    args = dict(block=(5, 5), output="centre", theta=0.05, dt=0.1, steps=500, m=30,
                name="heat2d-20x20")
    args.update(kw)
    return heat((20, 20), **args)


def heat3d_100(**kw) -> Problem:
    """100^3 grid, 10^3 heated corner block, mean of the 8 centre cells,
    unsafe y >= 0.01, dt 0.02, 1000 steps, Lanczos m = 40."""
    args = dict(block=(10, 10, 10), output="centre8", theta=0.01, dt=0.02, steps=1000,
                m=40, name="heat3d-100^3")
    args.update(kw)
    return heat((100, 100, 100), **args)


def heat3d_1000(**kw) -> Problem:
    """1000^3 grid (n = 1e9), 100^3 heated corner block, centre cell output,
    dt 0.02, 200 steps, Lanczos m = 30 (unsafe y >= 0.01)."""
    args = dict(block=(100, 100, 100), output="centre", theta=0.01, dt=0.02, steps=200,
                m=30, name="heat3d-1000^3")
    args.update(kw)
    return heat((1000, 1000, 1000), **args)


def heat3d_truncated(full: Problem, side: int) -> Problem:
    """The same heat problem on the sub-grid [0, side)^3 with the *same* h.

    A Krylov vector after j steps is supported within j stencil hops of the
    heated block, so while block + m < side - 1 the Lanczos coefficients and
    projections on the truncated grid equal those of the full grid (the far
    Dirichlet faces are never reached).  The output cell, if outside the
    sub-grid, is dropped (its projection is exactly 0 on the full grid too).
    """
    s = full.system
    dims = tuple(side for _ in s.dims)
    sysm = GridSystem(dims=dims, coef=s.coef, h=s.h)
    col = full.columns[0]
    return Problem(system=sysm, columns=[col], C_row_ptr=np.array([0, 0], dtype=np.int64),
                   C_col=np.zeros(0, dtype=np.int64), C_val=np.zeros(0), theta=np.array([math.inf]),
                   dt=full.dt, steps=full.steps, m=full.m, method=full.method,
                   precision=full.precision, name=full.name + f"-trunc{side}")


# --------------------------------------------------------------------------
# random sparse nonsymmetric system with forcing (stand-in for Sec. 5.1)
# --------------------------------------------------------------------------
def random_csr(n: int, nnz_per_row: int = 10, seed: int = 0, with_b: bool = True,
               column_dominant: bool = False) -> CsrSystem:
    """n x n, nnz_per_row distinct off-diagonal columns per row drawn uniformly
    (never the row itself), values N(0,1)/sqrt(nnz_per_row), diagonal
    -(row abs-sum + 0.1), or with column_dominant -(max(row, column abs-sum)
    + 0.1) (dominant in both directions); b ~ U[-0.01, 0.01]."""
    rng = np.random.default_rng(seed)
    k = nnz_per_row
    rows = np.arange(n, dtype=np.int64)
    off = rng.integers(0, n - 1, size=(n, k), dtype=np.int64)
    off = off + (off >= rows[:, None])
    off.sort(axis=1)
    while True:
        dup = np.any(off[:, 1:] == off[:, :-1], axis=1)
        if not dup.any():
            break
        bad = np.nonzero(dup)[0]
        redraw = rng.integers(0, n - 1, size=(len(bad), k), dtype=np.int64)
        redraw = redraw + (redraw >= bad[:, None])
        redraw.sort(axis=1)
        off[bad] = redraw
    vals = rng.standard_normal((n, k)) / math.sqrt(k)
    rsum = np.abs(vals).sum(axis=1)
    if column_dominant:
        csum = np.bincount(off.reshape(-1), weights=np.abs(vals).reshape(-1), minlength=n)
        rsum = np.maximum(rsum, csum)
    diag = -(rsum + 0.1)
    cols = np.concatenate([off, rows[:, None]], axis=1)
    allv = np.concatenate([vals, diag[:, None]], axis=1)
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    allv = np.take_along_axis(allv, order, axis=1)
    row_ptr = np.arange(n + 1, dtype=np.int64) * (k + 1)
    b = rng.uniform(-0.01, 0.01, size=n) if with_b else None
    return CsrSystem(n=n, row_ptr=row_ptr, col=cols.reshape(-1).astype(np.int32),
                     val=allv.reshape(-1).astype(np.float64), b=b, symmetric=False)


def random_csr_problem(n: int = 2_000_000, *, seed: int = 0, n_gen: int = 16, o: int = 2,
                       c_width: int = 1000, dt: float = 0.01, steps: int = 2000, m: int = 60,
                       theta: Optional[Sequence[float]] = None, precision: str = "fp64",
                       with_b: bool = True, name: str = "") -> Problem:
    """Box initial set on n_gen random variables each in [-1, 1] (one unit
    generator per variable) plus the fixed centre column (zero state, constant
    variable 1); C = o random +-1 rows over c_width distinct variables."""
    sysm = random_csr(n, seed=seed, with_b=with_b)
    return csr_problem_on(sysm, seed=seed, n_gen=n_gen, o=o, c_width=c_width, dt=dt, steps=steps, m=m,
                          theta=theta, precision=precision, name=name)


def csr_problem_on(sysm: CsrSystem, *, seed: int, n_gen: int = 16, o: int = 2, c_width: int = 1000,
                   dt: float = 0.01, steps: int = 2000, m: int = 60, theta: Optional[Sequence[float]] = None,
                   precision: str = "fp64", name: str = "") -> Problem:
    """The initial set and outputs of random_csr_problem on a given system."""
    n = sysm.n
    rng = np.random.default_rng(seed + 7919)
    gvars = rng.choice(n, size=n_gen, replace=False)
    cols = [Column(kind="sparse", zlo=-1.0, zhi=1.0, idx=np.array([v], dtype=np.int64),
                   val=np.array([1.0])) for v in gvars]
    cols.append(Column(kind="sparse", zlo=1.0, zhi=1.0, is_fixed=True,
                       idx=np.zeros(0, dtype=np.int64), val=np.zeros(0)))
    rows = []
    for _ in range(o):
        cidx = np.sort(rng.choice(n, size=min(c_width, n), replace=False))
        sgn = rng.choice([-1.0, 1.0], size=len(cidx))
        rows.append((cidx, sgn))
    rp, cc, cv = _c_rows(rows)
    th = np.full(o, math.inf) if theta is None else np.asarray(theta, dtype=np.float64)
    return Problem(system=sysm, columns=cols, C_row_ptr=rp, C_col=cc, C_val=cv, theta=th,
                   dt=dt, steps=steps, m=m, method="auto", precision=precision,
                   name=name or f"csr-{n}")


# --------------------------------------------------------------------------
# timed harmonic oscillator (Sec. 2.2)
# --------------------------------------------------------------------------
def oscillator(theta: float = 4.0) -> Problem:
    """x' = y, y' = -x, t' = 1 as x' = A x + b with b = (0, 0, 1).
    Initial set x0 = -5, y0 in [0, 1], t0 = 0: the fixed column (-5, 0, 0)
    carries the constant variable, the generator (0, 1, 0) has z in [0, 1].
    Output x, unsafe x >= theta, step pi/4, horizon pi (4 steps)."""
    A_rp = np.array([0, 1, 2, 2], dtype=np.int64)
    A_col = np.array([1, 0], dtype=np.int32)
    A_val = np.array([1.0, -1.0])
    sysm = CsrSystem(n=3, row_ptr=A_rp, col=A_col, val=A_val, b=np.array([0.0, 0.0, 1.0]),
                     symmetric=False)
    cols = [Column(kind="dense", zlo=0.0, zhi=1.0, dense=np.array([0.0, 1.0, 0.0])),
            Column(kind="dense", zlo=1.0, zhi=1.0, is_fixed=True, dense=np.array([-5.0, 0.0, 0.0]))]
    rp, cc, cv = _c_rows([([0], [1.0])])
    return Problem(system=sysm, columns=cols, C_row_ptr=rp, C_col=cc, C_val=cv,
                   theta=np.array([theta]), dt=math.pi / 4, steps=4, m=4, method="arnoldi",
                   name="oscillator")


def paper_heat_factors(N: int, coef: float = 0.01, exchange: float = 0.5):
    """The 1-D factors of the paper's heat model (Sec. 5.3: a unit cube,
    every face insulated except x = 1, which exchanges heat with the ambient
    (temperature 0) at constant `exchange`), discretised by cell-centred
    finite volumes: N cells of width h = 1/N per axis, coupling coef/h^2
    between neighbours, no flux through an insulated face.  At x = 1 the flux
    -coef u_x = exchange u_b runs through the half cell next to the face;
    eliminating the face value u_b leaves the last x-cell the diagonal term
    -g/h with g = exchange (2 coef/h) / (2 coef/h + exchange).  Returns
    (A_x, A_y, A_z) dense N x N: A = A_x (+) A_y (+) A_z (Kronecker sum, x
    fastest), symmetric and negative definite."""
    h = 1.0 / N
    L = np.zeros((N, N))
    for i in range(N - 1):
        L[i, i + 1] = L[i + 1, i] = 1.0
        L[i, i] -= 1.0
        L[i + 1, i + 1] -= 1.0
    Ay = (coef / h ** 2) * L
    Ax = Ay.copy()
    g = exchange * (2 * coef / h) / (2 * coef / h + exchange)
    Ax[N - 1, N - 1] -= g / h
    return Ax, Ay, Ay.copy()


def paper_heat(N: int = 100, *, dt: float = 0.02, steps: int = 1000, m: int = 800, err_target: float = 0.0,
               zlo: float = 0.9, zhi: float = 1.1, theta: float = math.inf, precision: str = "fp64",
               coef: float = 0.01, exchange: float = 0.5) -> Problem:
    """The paper's 3-D heat benchmark (Sec. 5.3) on N^3 cells: the model of
    paper_heat_factors as a symmetric CSR matrix (7 entries per interior
    row); the heated region x in [0, 0.4], y in [0, 0.2], z in [0, 0.1]
    (cells whose centres lie in it) at a temperature in [zlo, zhi], one
    column; the output is the temperature at the centre of the cube, the
    mean of the 8 cells around it; T = 20 by dt = 0.02 (1000 steps)."""
    import scipy.sparse as sp
    Ax, Ay, Az = paper_heat_factors(N, coef, exchange)
    I = sp.identity(N, format="csr")
    A = (sp.kron(sp.kron(I, I), sp.csr_matrix(Ax)) + sp.kron(sp.kron(I, sp.csr_matrix(Ay)), I)
         + sp.kron(sp.kron(sp.csr_matrix(Az), I), I)).tocsr()
    A.sort_indices()
    n = N ** 3
    sysm = CsrSystem(n=n, row_ptr=A.indptr.astype(np.int64), col=A.indices.astype(np.int32),
                     val=A.data.astype(np.float64), b=None, symmetric=True)
    centres = (np.arange(N) + 0.5) / N
    bx, by, bz = (int(np.sum(centres <= lim)) for lim in (0.4, 0.2, 0.1))
    ix = np.arange(bx)
    idx = (np.arange(bz)[:, None, None] * N * N + np.arange(by)[None, :, None] * N + ix[None, None, :]).ravel()
    col = Column(kind="sparse", zlo=zlo, zhi=zhi, idx=np.sort(idx).astype(np.int64), val=np.ones(idx.size))
    c = [N // 2 - 1, N // 2]
    cells = [(z * N + y) * N + x for z in c for y in c for x in c]
    rp, cc, cv = _c_rows([(cells, [0.125] * 8)])
    return Problem(system=sysm, columns=[col], C_row_ptr=rp, C_col=cc, C_val=cv, theta=np.array([theta]),
                   dt=dt, steps=steps, m=m, err_target=err_target, precision=precision,
                   name=f"paper-heat3d-{N}^3")


def paper_heat_exchange_face(N: int, coef: float = 0.01, exchange: float = 0.5) -> float:
    """The face coefficient of the x = 1 face of the paper's heat model on N
    cells per axis (Sec. 5.3, as in paper_heat_factors): g / h with
    g = exchange (2 coef/h) / (2 coef/h + exchange), h = 1/N."""
    h = 1.0 / N
    return exchange * (2 * coef / h) / (2 * coef / h + exchange) / h


def paper_heat_grid(N: int = 100, *, dt: float = 0.02, steps: int = 1000, m: int = 800, err_target: float = 0.0,
                    zlo: float = 0.9, zhi: float = 1.1, theta: float = math.inf, precision: str = "fp64",
                    coef: float = 0.01, exchange: float = 0.5) -> Problem:
    """paper_heat as a matrix-free grid system: N^3 cells of width h = 1/N,
    coupling coef/h^2, every face insulated (gamma = 0) except x = 1
    (gamma = paper_heat_exchange_face); the heated region as one box column
    (the cells whose centres lie in [0, 0.4] x [0, 0.2] x [0, 0.1]); the output
    the mean of the 8 cells around the centre.  The same operator, column and
    output as paper_heat."""
    h = 1.0 / N
    face = (0.0, paper_heat_exchange_face(N, coef, exchange), 0.0, 0.0, 0.0, 0.0)
    sysm = GridSystem(dims=(N, N, N), coef=coef, h=(h, h, h), face=face)
    centres = (np.arange(N) + 0.5) / N
    bx, by, bz = (int(np.sum(centres <= lim)) for lim in (0.4, 0.2, 0.1))
    col = Column(kind="box", zlo=zlo, zhi=zhi, box_lo=(0, 0, 0), box_hi=(bx, by, bz), value=1.0)
    c = [N // 2 - 1, N // 2]
    cells = [(z * N + y) * N + x for z in c for y in c for x in c]
    rp, cc, cv = _c_rows([(cells, [0.125] * 8)])
    return Problem(system=sysm, columns=[col], C_row_ptr=rp, C_col=cc, C_val=cv, theta=np.array([theta]),
                   dt=dt, steps=steps, m=m, err_target=err_target, precision=precision,
                   name=f"paper-heat3d-grid-{N}^3")


def replicated_blocks(h: int, *, seed: int = 0, dt: float = 0.1, steps: int = 300, m: int = 28,
                      theta: float = 0.45, precision: str = "fp64", simulate: str = "auto") -> Problem:
    """The replicated-helicopter shape of Sec. 5.2 with a stand-in block: the
    28-dimensional helicopter model is not available, so one seeded random
    stable 28 x 28 block B (entries N(0,1)/sqrt(28), shifted so that its
    rightmost eigenvalue has real part -0.05) is copied h times on the
    diagonal, n = 28 h.  Eight variables of every copy (its first eight) are
    intervals [0.9, 1.1] * (their seeded base value in [0.1, 0.3]), so i = 8 h unit
    generators; the output is the mean of the eighth variable over the copies
    (o = 1), unsafe above theta; horizon 30 at step 0.1 (300 steps)."""
    rng = np.random.default_rng(seed + 2828)
    B = rng.standard_normal((28, 28)) / math.sqrt(28)
    B -= (np.max(np.linalg.eigvals(B).real) + 0.05) * np.eye(28)
    base = rng.uniform(0.1, 0.3, 8)
    nzr, nzc = np.nonzero(B)
    vals_b = B[nzr, nzc]
    per = len(vals_b)
    n = 28 * h
    offs = (np.arange(h, dtype=np.int64) * 28)[:, None]
    rows = (offs + nzr[None, :]).reshape(-1)
    cols = (offs + nzc[None, :]).reshape(-1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    sysm = CsrSystem(n=n, row_ptr=row_ptr, col=cols.astype(np.int32), val=np.tile(vals_b, h).astype(np.float64),
                     b=None, symmetric=False)
    cols_e = []
    for k in range(h):
        for v in range(8):
            cols_e.append(Column(kind="sparse", zlo=0.9 * base[v], zhi=1.1 * base[v],
                                 idx=np.array([28 * k + v], dtype=np.int64), val=np.array([1.0])))
    rp, cc, cv = _c_rows([(np.arange(h, dtype=np.int64) * 28 + 7, np.full(h, 1.0 / h))])
    assert per * h == len(sysm.val)
    return Problem(system=sysm, columns=cols_e, C_row_ptr=rp, C_col=cc, C_val=cv, theta=np.array([theta]),
                   dt=dt, steps=steps, m=m, precision=precision, simulate=simulate,
                   name=f"replicated-blocks-h{h}")


# --------------------------------------------------------------------------
# small random cases
# --------------------------------------------------------------------------
def random_symmetric_csr(n: int, nnz_per_row: int = 4, seed: int = 0) -> CsrSystem:
    """Symmetric negative-definite sparse A = -(B + B^T)/2 - shift*I style:
    random symmetric off-diagonal pattern, diagonal -(row abs-sum + 0.5)."""
    rng = np.random.default_rng(seed)
    pairs = set()
    for r in range(n):
        for c in rng.choice(n, size=min(nnz_per_row, n - 1), replace=False):
            if c != r:
                pairs.add((min(r, int(c)), max(r, int(c))))
    dense = np.zeros((n, n))
    for (r, c) in pairs:
        v = rng.standard_normal() / math.sqrt(nnz_per_row)
        dense[r, c] = v
        dense[c, r] = v
    dense[np.diag_indices(n)] = -(np.abs(dense).sum(axis=1) + 0.5)
    return dense_to_csr(dense, symmetric=True)


def dense_to_csr(dense: np.ndarray, b: Optional[np.ndarray] = None, symmetric: bool = False) -> CsrSystem:
    n = dense.shape[0]
    rp = [0]
    cols: List[int] = []
    vals: List[float] = []
    for r in range(n):
        nz = np.nonzero(dense[r])[0]
        cols.extend(int(c) for c in nz)
        vals.extend(float(dense[r, c]) for c in nz)
        rp.append(len(cols))
    return CsrSystem(n=n, row_ptr=np.asarray(rp, dtype=np.int64), col=np.asarray(cols, dtype=np.int32),
                     val=np.asarray(vals, dtype=np.float64), b=b, symmetric=symmetric)


def random_problem(sysm, *, seed: int, n_cols: int = 2, o: int = 2, dt: float = 0.05,
                   steps: int = 40, m: int = 10, theta=None, fixed_last: bool = False,
                   method: str = "auto", precision: str = "fp64") -> Problem:
    """Random dense columns and dense random output rows for small systems."""
    rng = np.random.default_rng(seed)
    n = sysm.n
    cols = []
    for j in range(n_cols):
        fixed = fixed_last and j == n_cols - 1
        lo, hi = (1.0, 1.0) if fixed else (float(-rng.uniform(0, 1)), float(rng.uniform(0, 1)))
        cols.append(Column(kind="dense", zlo=lo, zhi=hi, is_fixed=fixed, dense=rng.standard_normal(n)))
    rows = [(np.arange(n), rng.standard_normal(n)) for _ in range(o)]
    rp, cc, cv = _c_rows(rows)
    th = np.full(o, math.inf) if theta is None else np.asarray(theta, dtype=np.float64)
    return Problem(system=sysm, columns=cols, C_row_ptr=rp, C_col=cc, C_val=cv, theta=th,
                   dt=dt, steps=steps, m=m, method=method, precision=precision,
                   name=f"random-{n}-{seed}")


def column_dense(col: Column, n: int, dims: Optional[Sequence[int]] = None) -> np.ndarray:
    """Materialise one column as a dense vector (input handling only)."""
    v = np.zeros(n)
    if col.kind == "dense":
        v[:] = col.dense
    elif col.kind == "sparse":
        v[np.asarray(col.idx, dtype=np.int64)] = col.val
    elif col.kind == "box":
        assert dims is not None
        sl = tuple(slice(lo, hi) for lo, hi in zip(reversed(col.box_lo), reversed(col.box_hi)))
        v.reshape(tuple(reversed(dims)))[sl] = col.value
    else:
        raise ValueError(col.kind)
    return v


# --------------------------------------------------------------------------
# serving stream
# --------------------------------------------------------------------------
def serving_mix(n_queries: int = 512, seed: int = 0, *, side2d=(100, 2000), side3d=(100, 400),
                csr_n=(100_000, 2_000_000), csr_sizes: int = 5, gens=(1, 32), steps=(100, 2000), m=(20, 60),
                precision: str = "fp32", heat_precision: str = "fp64", simulate: str = "auto") -> List[Problem]:
    """A seeded mix of verification queries, one third each:
      * 2D heat, side log-uniform in side2d (n = side^2), block side/4, dt 0.1;
      * 3D heat, side log-uniform in side3d, block side/10, dt 0.02;
      (heat outputs: the cell just past the block's far corner, so that every
      query's projected output is nonzero, the grid centre being out of the
      Krylov space's reach at these m; storage `heat_precision`);
      * random CSR systems of random_csr (sizes log-spaced in csr_n, `csr_sizes`
        distinct systems shared by the queries), `gens` unit generators plus the
        fixed column, two +-1 output rows, dt 0.01;
    horizons uniform in `steps`, Krylov dimension uniform in `m`, thresholds +inf;
    `simulate` for every query ("auto": the transpose dynamics where o < i).
    """
    rng = np.random.default_rng(seed + 4242)
    sizes = sorted(set(int(round(x)) for x in np.geomspace(csr_n[0], csr_n[1], csr_sizes)))
    cache: dict = {}
    out: List[Problem] = []
    for q in range(n_queries):
        kind = int(rng.integers(3))
        st = int(rng.integers(steps[0], steps[1] + 1))
        mm = int(rng.integers(m[0], m[1] + 1))
        if kind == 0:
            side = int(round(math.exp(rng.uniform(math.log(side2d[0]), math.log(side2d[1])))))
            b = max(side // 4, 1)
            out.append(heat((side, side), block=(b, b), output="edge", dt=0.1, steps=st, m=mm,
                            precision=heat_precision, name=f"q{q}-heat2d-{side}"))
        elif kind == 1:
            side = int(round(math.exp(rng.uniform(math.log(side3d[0]), math.log(side3d[1])))))
            b = max(side // 10, 1)
            out.append(heat((side, side, side), block=(b, b, b), output="edge", dt=0.02, steps=st, m=mm,
                            precision=heat_precision, name=f"q{q}-heat3d-{side}"))
        else:
            n = sizes[int(rng.integers(len(sizes)))]
            if n not in cache:
                cache[n] = random_csr(n, seed=1000 + len(cache))
            g = int(rng.integers(gens[0], gens[1] + 1))
            out.append(csr_problem_on(cache[n], seed=q, n_gen=g, o=2, c_width=min(1000, n // 4), dt=0.01,
                                      steps=st, m=mm, precision=precision, name=f"q{q}-csr-{n}-g{g}"))
        out[-1].simulate = simulate
    return out
