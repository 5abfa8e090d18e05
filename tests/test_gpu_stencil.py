"""Parity of the CUDA grid-Laplacian Lanczos path against the CPU oracle.

FP64 form: every bound within 1e-9 (scale-normalised), identical first
violation step and row, H and P within 1e-9.  FP32-storage form: bounds within
1e-6 of the FP64 oracle, identical violation step.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from parity import bound_error, check_violation, krylov_error, margin_ok

pytestmark = pytest.mark.gpu

kv = pytest.importorskip("paper_1804_01583_gb300")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_01583_gb300 import build as kvbuild
    kvbuild.build()
    c = kv.Context(40 << 30)
    yield c
    c.close()


def run_gpu(ctx, p, **kw):
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p, **kw)
    try:
        return ph.run()
    finally:
        ph.close()
        sysh.close()


def check_fp64(ctx, p, tol=1e-9, **kw):
    got = run_gpu(ctx, p, **kw)
    ref = oracle.run(p)
    for j in range(p.i):
        eh, ep = krylov_error(got, ref, j)
        assert eh <= tol and ep <= tol, (j, eh, ep)
        assert abs(got["beta0"][j] - ref["beta0"][j]) <= 1e-14 * max(ref["beta0"][j], 1e-300)
    e = bound_error(got, ref)
    assert e <= tol, e
    assert margin_ok(ref, p)
    check_violation(got, ref, p, tol)
    return got, ref


@pytest.mark.parametrize("expm_mode", ["per_step", "propagate"])
@pytest.mark.parametrize("theta", [0.05, 0.01])
def test_heat2d_20x20(ctx, expm_mode, theta):
    """20x20 grid, 5x5 heated block, centre output, 500 steps, m = 30; the
    unsafe threshold 0.05 is never reached, 0.01 is (violation variant)."""
    p = W.heat2d_20(theta=theta)
    got, ref = check_fp64(ctx, p, expm_mode=expm_mode)
    if theta == 0.01:
        assert ref["viol_step"] > 0
    else:
        assert ref["viol_step"] == -1


def test_ragged_3d_grid(ctx):
    """Extents that are not multiples of the 32 x 8 thread tile or the z chunk."""
    p = W.heat((37, 19, 23), block=(5, 4, 3), output="centre8", theta=math.inf, dt=0.01, steps=120, m=25)
    check_fp64(ctx, p)


@pytest.mark.parametrize("dims,block", [((3, 3), (1, 1)), ((4, 4), (4, 4)), ((2, 3, 2), (1, 1, 1))])
def test_breakdown_on_tiny_grids(ctx, dims, block):
    """The Krylov space is exhausted before m = 30 steps (n = 9, or a
    symmetric start vector on 16 cells): both sides stop at the same step and
    the result is exact."""
    p = W.heat(dims, block=block, output="centre", dt=0.05, steps=40, m=30)
    got, ref = check_fp64(ctx, p)
    assert ref["used"][0] < 30


def test_heat3d_100_full(ctx):
    """100^3 grid, 10^3 corner block, mean of the 8 centre cells, m = 40,
    1000 steps: the output cell is 120 stencil hops from the block, so the
    projected Krylov output is exactly 0 on both sides; the tridiagonal H is
    compared to 1e-9."""
    p = W.heat3d_100()
    got, ref = check_fp64(ctx, p)
    assert np.all(ref["hi"] == 0.0)


def test_heat3d_100_output_within_reach(ctx):
    """Same grid and initial set with an output cell 9 hops away, so the bounds
    are non-zero at full size."""
    p = W.heat3d_100(m=40, steps=400)
    cell = W.grid_index((100, 100, 100), (12, 12, 12))
    p.C_row_ptr = np.array([0, 1], dtype=np.int64)
    p.C_col = np.array([cell], dtype=np.int64)
    p.C_val = np.array([1.0])
    p.theta = np.array([0.05])
    got, ref = check_fp64(ctx, p)
    assert np.max(ref["hi"]) > 0


def test_sparse_dense_and_multi_columns(ctx):
    """Columns given as a point source, a dense random field and a box, with two
    output rows (one dense-ish): init through scatter / dense copy kernels."""
    dims = (24, 17, 9)
    n = 24 * 17 * 9
    rng = np.random.default_rng(3)
    sysm = W.GridSystem(dims=dims, coef=0.01, h=tuple(1.0 / (d + 1) for d in dims))
    cols = [W.Column(kind="sparse", zlo=-1.0, zhi=2.0, idx=np.array([W.grid_index(dims, (3, 4, 5))]),
                     val=np.array([1.0])),
            W.Column(kind="dense", zlo=0.0, zhi=0.5, dense=rng.standard_normal(n)),
            W.Column(kind="box", zlo=0.9, zhi=1.1, box_lo=(0, 0, 0), box_hi=(4, 3, 2), value=2.0)]
    rp, cc, cv = W._c_rows([([W.grid_index(dims, (6, 6, 4))], [1.0]),
                            (np.arange(0, n, 7), rng.standard_normal(len(range(0, n, 7))))])
    p = W.Problem(system=sysm, columns=cols, C_row_ptr=rp, C_col=cc, C_val=cv,
                  theta=np.array([math.inf, math.inf]), dt=0.02, steps=80, m=20)
    check_fp64(ctx, p)


def test_zero_column(ctx):
    p = W.heat((10, 10), block=(3, 3), output="centre", dt=0.1, steps=10, m=5)
    p.columns[0].value = 0.0
    got = run_gpu(ctx, p)
    assert got["m_used"][0] == 0 and np.all(got["hi"] == 0) and np.all(got["lo"] == 0)


def test_deterministic(ctx):
    p = W.heat((37, 19, 23), block=(5, 4, 3), output="centre8", dt=0.01, steps=50, m=25)
    a = run_gpu(ctx, p)
    b = run_gpu(ctx, p)
    assert np.array_equal(a["H"], b["H"]) and np.array_equal(a["hi"], b["hi"])


PATHS = {"fused": 0, "two_pass": 1}  # 1 = KV_FLAG_TWO_PASS


@pytest.mark.parametrize("path", ["fused", "two_pass"])
@pytest.mark.parametrize("theta", [0.05, 0.01])
def test_fp32_storage_heat2d(ctx, theta, path):
    """FP32 vectors, error-free float dot products summed in double: bounds
    within 1e-6 of the FP64 oracle and the same violation step, through the
    single-pass TMA iteration and through the two-pass kernels."""
    p = W.heat2d_20(theta=theta, precision="fp32")
    got = run_gpu(ctx, p, flags=PATHS[path])
    ref = oracle.run(W.heat2d_20(theta=theta))
    e = bound_error(got, ref)
    assert e <= 1e-6, e
    assert got["viol_step"] == ref["viol_step"]


@pytest.mark.parametrize("dims", [(37, 19, 23), (36, 19, 23), (260, 33, 40)])
@pytest.mark.parametrize("path", ["fused", "two_pass"])
def test_fp32_storage_3d(ctx, dims, path):
    """Partial tiles in x, y and z (the fused path needs nx % 4 == 0 and falls
    back to the two-pass kernels otherwise)."""
    kw = dict(block=(5, 4, 3), output="centre8", dt=0.01, steps=120, m=25)
    got = run_gpu(ctx, W.heat(dims, precision="fp32", **kw), flags=PATHS[path])
    ref = oracle.run(W.heat(dims, **kw))
    e = bound_error(got, ref)
    assert e <= 1e-6, e
    for j in range(1):
        eh, _ = krylov_error(got, ref, j)
        assert eh <= 1e-5, eh


@pytest.mark.parametrize("dims", [(132, 19, 9),     # 1 full-width tile + narrow tiles of 4 lanes per row pair
                                  (268, 70, 7),     # remainder 20: 8 lanes per row pair, two narrow y tiles
                                  (172, 33, 6),     # remainder 48: 16 lanes per row pair
                                  (224, 20, 5),     # remainder 100: one more full-width tile
                                  (20, 300, 4),     # narrow tiles only, five of them in y
                                  (1000, 40)])      # 2-D, 8 full-width tiles + a narrow one
def test_fp32_fused_tile_shapes(ctx, dims):
    """The single-pass iteration on every tile shape its grid plan uses (full
    width, narrow of 4, 8 or 16 lanes per row pair, ragged full width), with
    an initial block covering all but the last three cells of every axis, so
    every tile sees non-zero data and the centre output is well inside it:
    H within 1e-5 and bounds within 1e-6 of the FP64 oracle."""
    block = tuple(max(1, d - 3) for d in dims)
    kw = dict(block=block, output="centre8", dt=1e-4, steps=60, m=20)
    got = run_gpu(ctx, W.heat(dims, precision="fp32", **kw))
    ref = oracle.run(W.heat(dims, **kw))
    eh, _ = krylov_error(got, ref, 0)
    assert eh <= 1e-5, eh
    e = bound_error(got, ref)
    assert e <= 1e-6, e


@pytest.mark.parametrize("path", ["fused", "two_pass"])
def test_fp32_output_within_reach_100(ctx, path):
    """100^3 with a nearby output cell: non-zero bounds at full size in FP32."""
    p = W.heat3d_100(m=40, steps=400, precision="fp32")
    cell = W.grid_index((100, 100, 100), (12, 12, 12))
    for q in (p,):
        q.C_row_ptr = np.array([0, 1], dtype=np.int64)
        q.C_col = np.array([cell], dtype=np.int64)
        q.C_val = np.array([1.0])
        q.theta = np.array([0.05])
    got = run_gpu(ctx, p, flags=PATHS[path])
    p64 = W.heat3d_100(m=40, steps=400)
    p64.C_row_ptr, p64.C_col, p64.C_val, p64.theta = p.C_row_ptr, p.C_col, p.C_val, p.theta
    ref = oracle.run(p64)
    assert bound_error(got, ref) <= 1e-6
    assert got["viol_step"] == ref["viol_step"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_heat3d_1000_full_size(ctx, precision):
    """n = 1e9 (1000^3), 100^3 block, m = 30: the configuration the benchmark
    times.  After j steps the Krylov vector is supported within j hops of the
    block, so the same Lanczos run on a 140^3 sub-grid with the same h gives the
    same coefficients (support argument, pinned on the CPU in the oracle
    tests); the centre output is 400 hops away and exactly 0."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    need = (24 if precision == "fp64" else 12) << 30  # three vectors (single-pass form)
    if free < need + (2 << 30):
        pytest.skip("not enough device memory")
    p = W.heat3d_1000(precision=precision)
    got = run_gpu(ctx, p)
    ref = oracle.run(W.heat3d_truncated(W.heat3d_1000(), 140))
    mu = int(ref["used"][0])
    assert int(got["m_used"][0]) == mu == 30
    Hr = ref["H"][0][: mu + 1, :mu]
    Hg = got["H"][0][: mu + 1, :mu]
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert np.max(np.abs(Hg - Hr)) <= tol * np.max(np.abs(Hr))
    assert abs(got["beta0"][0] - ref["beta0"][0]) <= 1e-12 * ref["beta0"][0]
    assert np.all(got["P"] == 0.0) and np.all(got["hi"] == 0.0) and np.all(got["lo"] == 0.0)
    assert got["viol_step"] == -1


def test_invalid_arguments(ctx):
    p = W.heat2d_20()
    sysh = kv.System(ctx, p.system)
    for mutate in [lambda q: setattr(q, "m", 0), lambda q: setattr(q, "m", kv.KV_MAX_M_LANCZOS + 1),
                   lambda q: setattr(q, "dt", -1.0), lambda q: setattr(q, "steps", -2),
                   lambda q: setattr(q.columns[0], "box_hi", (21, 5)),
                   lambda q: setattr(q, "C_col", np.array([400], dtype=np.int64)),
                   lambda q: setattr(q, "method", "arnoldi")]:
        q = W.heat2d_20()
        mutate(q)
        with pytest.raises(kv.KvError) as ei:
            kv.ProblemHandle(ctx, sysh, q)
        assert ei.value.code == kv.KV_EINVAL
    sysh.close()


def test_pool_exhaustion_is_reported(ctx):
    """A problem that does not fit the context pool fails with KV_ENOMEM
    (admission by budget, not by allocating until the device fails)."""
    small = kv.Context(8 << 20)
    p = W.heat((200, 200, 200), block=(4, 4, 4), output="centre", dt=0.1, steps=5, m=5)
    sysh = kv.System(small, p.system)
    with pytest.raises(kv.KvError) as ei:
        kv.ProblemHandle(small, sysh, p)
    assert ei.value.code == kv.KV_ENOMEM
    assert small.pool_stats()[0] == 0
    sysh.close()
    small.close()


@pytest.mark.parametrize("precision,flags", [("fp64", 0), ("fp32", 0), ("fp32", 1)])
def test_many_output_rows(ctx, precision, flags):
    """40 output rows (more than the rows a finishing block projects itself):
    the projection of every new Krylov vector runs as its own grid kernel."""
    dims = (40, 36, 20)
    rng = np.random.default_rng(17)
    p = W.heat(dims, block=(10, 9, 5), output="centre8", dt=0.02, steps=60, m=30, precision=precision)
    rows = []
    for _ in range(40):
        cells = rng.choice(int(np.prod(dims)), size=5, replace=False)
        rows.append((np.sort(cells), rng.standard_normal(5)))
    p.C_row_ptr, p.C_col, p.C_val = W._c_rows(rows)
    p.theta = np.full(40, math.inf)
    got = run_gpu(ctx, p, flags=flags)
    p64 = W.heat(dims, block=(10, 9, 5), output="centre8", dt=0.02, steps=60, m=30)
    p64.C_row_ptr, p64.C_col, p64.C_val, p64.theta = p.C_row_ptr, p.C_col, p.C_val, p.theta
    ref = oracle.run(p64)
    tol = 1e-9 if precision == "fp64" else 1e-6
    assert bound_error(got, ref) <= tol
    if precision == "fp64":
        eh, ep = krylov_error(got, ref, 0)
        assert eh <= 1e-9 and ep <= 1e-9
