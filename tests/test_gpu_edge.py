"""Degenerate and extreme inputs against the oracle: a horizon of zero steps
(only t = 0: the bounds are C E z itself), Krylov dimension 1, an output row
without entries, a system of one variable with a forcing term (closed form
x0 e^{at} + (b/a)(e^{at} - 1)), and the largest Krylov dimensions of each
method (Arnoldi KV_MAX_M; Lanczos far above the shared-memory exponential)."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity import bound_error

pytestmark = pytest.mark.gpu

kv = pytest.importorskip("paper_1804_01583_gb300")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_01583_gb300 import build as kvbuild
    kvbuild.build()
    c = kv.Context(8 << 30)
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


def grid_inside(steps, m, precision="fp64"):
    """A 3-D grid whose heated corner block covers the centre cell, so the
    output at t = 0 is the block temperature."""
    return W.heat((12, 10, 8), block=(8, 6, 5), output="centre", dt=0.05, steps=steps, m=m, precision=precision)


def csr_case(steps, m, o=2):
    return W.random_csr_problem(600, seed=11, n_gen=3, o=o, c_width=40, dt=0.01, steps=steps, m=m)


@pytest.mark.parametrize("case", ["grid_fp64", "grid_fp32", "csr"])
def test_zero_steps(ctx, case):
    p = {"grid_fp64": lambda: grid_inside(0, 10), "grid_fp32": lambda: grid_inside(0, 10, "fp32"),
         "csr": lambda: csr_case(0, 8)}[case]()
    got = run_gpu(ctx, p)
    ref = oracle.run(W.heat((12, 10, 8), block=(8, 6, 5), output="centre", dt=0.05, steps=0, m=10)
                     if case.startswith("grid") else p)
    assert got["hi"].shape == (p.o, 1)
    assert np.allclose(got["hi"], ref["hi"], rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(ref["hi"]))))
    assert np.allclose(got["lo"], ref["lo"], rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(ref["lo"]))))
    if case.startswith("grid"):
        assert got["hi"][0, 0] == pytest.approx(1.1) and got["lo"][0, 0] == pytest.approx(0.9)


@pytest.mark.parametrize("case", ["grid", "csr_arnoldi", "csr_lanczos"])
def test_krylov_dimension_one(ctx, case):
    if case == "grid":
        p = grid_inside(20, 1)
    elif case == "csr_arnoldi":
        p = csr_case(20, 1)
    else:
        p = W.random_problem(W.random_symmetric_csr(400, seed=12), seed=13, n_cols=2, o=1, dt=0.05, steps=20, m=1)
    got = run_gpu(ctx, p)
    ref = oracle.run(p)
    assert all(int(got["m_used"][j]) == int(ref["used"][j]) == 1 for j in range(p.i))
    assert bound_error(got, ref) <= 1e-12


def test_empty_output_row(ctx):
    """The first output row has no entries: its bounds are exactly zero; the
    second row is unaffected."""
    p = csr_case(30, 12)
    p.C_row_ptr = np.array([0, 0, p.C_row_ptr[1]], dtype=np.int64)
    p.C_col = p.C_col[:p.C_row_ptr[2]]
    p.C_val = p.C_val[:p.C_row_ptr[2]]
    p.theta = np.array([0.0, np.inf])          # 0 >= 0: the empty row violates at step 0
    got = run_gpu(ctx, p)
    ref = oracle.run(p)
    assert np.all(got["hi"][0] == 0.0) and np.all(got["lo"][0] == 0.0)
    assert bound_error(got, ref) <= 1e-9
    assert got["viol_step"] == ref["viol_step"] == 0 and got["viol_row"] == 0


def test_one_variable_system(ctx):
    """x' = -x/2 + 0.2, x0 in [0.5, 1.5]: one generator and the fixed column
    (the constant) on the 2-variable augmented system."""
    s1 = W.CsrSystem(n=1, row_ptr=np.array([0, 1], dtype=np.int64), col=np.array([0], dtype=np.int32),
                     val=np.array([-0.5]), b=np.array([0.2]))
    rp, cc, cv = W._c_rows([([0], [1.0])])
    cols = [W.Column(kind="dense", zlo=0.5, zhi=1.5, dense=np.array([1.0])),
            W.Column(kind="dense", zlo=1.0, zhi=1.0, is_fixed=True, dense=np.array([0.0]))]
    p = W.Problem(system=s1, columns=cols, C_row_ptr=rp, C_col=cc, C_val=cv, theta=np.array([1.2]),
                  dt=0.5, steps=8, m=2)
    got = run_gpu(ctx, p)
    ref = oracle.run(p)
    t = p.dt * np.arange(p.steps + 1)
    e = np.exp(-0.5 * t)
    assert np.allclose(got["hi"][0], 1.5 * e + 0.4 * (1 - e), rtol=0, atol=1e-12)
    assert np.allclose(got["lo"][0], 0.5 * e + 0.4 * (1 - e), rtol=0, atol=1e-12)
    assert got["viol_step"] == ref["viol_step"] == 0          # 1.5 >= 1.2 at t = 0
    assert bound_error(got, ref) <= 1e-12


def test_arnoldi_at_the_largest_dimension(ctx):
    """m = KV_MAX_M (256) Arnoldi iterations on a 300-variable system with
    forcing: the basis rows and bounds within 1e-9 (both sides converged)."""
    p = W.random_csr_problem(300, seed=14, n_gen=2, o=1, c_width=50, dt=0.01, steps=3, m=kv.KV_MAX_M)
    got = run_gpu(ctx, p)
    ref = oracle.run(p)
    for j in range(p.i):
        assert int(got["m_used"][j]) == int(ref["used"][j])
        S = max(np.max(np.abs(ref["basis"][j])), 1e-300)
        assert np.max(np.abs(got["basis"][j] - ref["basis"][j])) <= 1e-9 * S
    assert bound_error(got, ref) <= 1e-9


def test_lanczos_far_above_the_shared_memory_exponential(ctx):
    """m = 400 Lanczos iterations on a 30 x 30 grid (n = 900), the
    global-memory exponential at m = 400: the basis rows and bounds within
    1e-9.  H and P are not compared: without reorthogonalisation (Alg. 3)
    converged Ritz values spawn ghost copies at iterations that depend on
    rounding, so the two sides' H drift apart (by O(1) here) while the
    converged output C V e^{tH} e_1 does not."""
    p = W.heat((30, 30), block=(4, 4), output="centre", dt=0.5, steps=3, m=400)
    got = run_gpu(ctx, p)
    ref = oracle.run(p)
    assert int(got["m_used"][0]) == int(ref["used"][0])
    S = np.max(np.abs(ref["basis"][0]))
    assert np.max(np.abs(got["basis"][0] - ref["basis"][0])) <= 1e-9 * S
    assert bound_error(got, ref) <= 1e-9


def test_grid_without_coupling(ctx):
    """coef = 0: A = 0 and the outputs stay C E z at every step (the Krylov
    space breaks down after one vector), against the oracle; the grid runs
    the single-pass FP64 kernel in its plain form (the unit form divides by
    kappa_x = 0).  Face coefficients with coef = 0 are refused: the kernels
    hold a face as its share of the coupling it replaces."""
    dims = (16, 16, 20)
    sysm = W.GridSystem(dims=dims, coef=0.0, h=(0.1, 0.1, 0.1))
    base = W.heat(dims, block=(6, 4, 3), output="centre", dt=0.05, steps=20, m=8)
    cell = W.grid_index(dims, (dims[0] - 1, 2, 1))
    rp, cc, cv = W._c_rows([([cell, W.grid_index(dims, (3, 2, 1))], [1.0, 1.0])])
    col = W.Column(kind="box", zlo=0.5, zhi=1.5, box_lo=(2, 0, 0), box_hi=(dims[0], 6, 4), value=1.0)
    p = W.Problem(**{**base.__dict__, "system": sysm, "columns": [col], "C_row_ptr": rp, "C_col": cc,
                     "C_val": cv, "theta": np.array([np.inf])})
    got = run_gpu(ctx, p)
    assert bound_error(got, oracle.run(p)) <= 1e-9
    assert np.allclose(got["hi"], 3.0) and np.allclose(got["lo"], 1.0)
    faced = W.GridSystem(dims=dims, coef=0.0, h=(0.1, 0.1, 0.1), face=(0.0, 3.0, 0.0, 0.0, 0.0, 0.0))
    with pytest.raises(kv.KvError) as ei:
        kv.System(ctx, faced)
    assert ei.value.code == kv.KV_EINVAL and "coef > 0" in str(ei.value)
