"""Parity of the transpose-dynamics simulation on the GPU (Sec. 4.1: one
Krylov run per output row on A^T or A'^T, projected by E'^T, the basis
transposed back) against the oracle's transposed path: basis rows and bounds
within 1e-9 (FP64) / 1e-6 (FP32 storage), identical violation step; Lanczos
runs also H and P."""
import json
import os

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
    c = kv.Context(32 << 30)
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


def basis_error(got, ref, p):
    S = max(np.max(np.abs(ref["basis"][j])) for j in range(p.i))
    if S == 0.0:
        return float(np.max(np.abs(got["basis"])))
    return max(float(np.max(np.abs(got["basis"][j] - ref["basis"][j]))) for j in range(p.i)) / S


def check(got, ref, p, tol, lanczos):
    assert got["transposed"]
    for r in range(p.o):
        assert int(got["m_used"][r]) == int(ref["used"][r]), (r, got["m_used"][r], ref["used"][r])
        if lanczos:
            eh, ep = krylov_error(got, ref, r)
            assert eh <= tol and ep <= tol, (r, eh, ep)
    assert basis_error(got, ref, p) <= tol
    assert bound_error(got, ref) <= tol


@pytest.mark.parametrize("expm_mode", ["per_step", "propagate"])
def test_oscillator_transposed(ctx, golden_dir, expm_mode):
    """Sec. 4.1: one run of the transpose dynamics gives the basis row
    (0.707, 3.54) at 3 pi / 4 and the violation at step 3."""
    g = json.load(open(os.path.join(golden_dir, "oscillator.json")))
    p = W.oscillator()
    p.simulate = "transpose"
    got = run_gpu(ctx, p, expm_mode=expm_mode)
    ref = oracle.run(p)
    k = g["violation_step"]
    assert got["viol_step"] == k and len(got["m_used"]) == 1
    assert abs(got["basis"][0][0, k] - g["basis_at_violation"]["i_y"]) < g["printed_digits_tol"]
    assert abs(got["basis"][1][0, k] - g["basis_at_violation"]["i_f"]) < g["printed_digits_tol"]
    check(got, ref, p, 1e-9, False)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_random_csr_with_forcing_transposed(ctx, precision):
    """The 16-generator random-CSR workload at n = 2e4 (i = 17 with the fixed
    column, o = 2, m = 60): 2 Arnoldi runs on A'^T instead of 17 on A', with
    a violating threshold."""
    mk = lambda prec: W.random_csr_problem(20000, seed=0, m=60, steps=2000, precision=prec)
    p64 = mk("fp64")
    p64.simulate = "transpose"
    ref = oracle.run(p64)
    p64.theta = 0.5 * np.max(ref["hi"], axis=1)
    ref = oracle.run(p64)
    assert ref["viol_step"] >= 0 and margin_ok(ref, p64)
    p = mk(precision)
    p.simulate, p.theta = "transpose", p64.theta
    got = run_gpu(ctx, p, expm_mode="propagate")
    tol = 1e-9 if precision == "fp64" else 1e-6
    check(got, ref, p64, tol, False)
    assert got["viol_step"] == ref["viol_step"]
    if precision == "fp64":
        check_violation(got, ref, p64, tol)


def test_symmetric_csr_lanczos_transposed(ctx):
    sysm = W.random_symmetric_csr(800, seed=3)
    p = W.random_problem(sysm, seed=4, n_cols=6, o=2, dt=0.05, steps=100, m=30)
    p.simulate = "transpose"
    got = run_gpu(ctx, p)
    ref = oracle.run(p)
    check(got, ref, p, 1e-9, True)


def test_grid_transposed_multi_column(ctx):
    """A grid with a box, a dense and a sparse column and one output row: one
    Lanczos run on the grid from the output row, projected by E^T."""
    dims = (24, 20, 12)
    n = int(np.prod(dims))
    rng = np.random.default_rng(5)
    p = W.heat(dims, block=(6, 5, 4), output="centre8", dt=0.02, steps=80, m=40)
    p.columns.append(W.Column(kind="dense", zlo=-0.5, zhi=0.5, dense=rng.standard_normal(n)))
    p.columns.append(W.Column(kind="sparse", zlo=0.0, zhi=2.0, idx=np.array([5, 777, 3000]),
                              val=np.array([1.0, -2.0, 0.5])))
    p.simulate = "auto"                      # o = 1 < i = 3
    got = run_gpu(ctx, p)
    ref = oracle.run(p)
    check(got, ref, p, 1e-9, True)
    # FP32 storage through the single-pass grid iteration
    p.precision = "fp32"
    got32 = run_gpu(ctx, p)
    assert basis_error(got32, ref, p) <= 1e-6 and bound_error(got32, ref) <= 1e-6


def test_transposed_error_control(ctx):
    from test_gpu_errbound import pick_target
    sysm = W.random_symmetric_csr(1500, seed=6)
    p = W.random_problem(sysm, seed=7, n_cols=5, o=2, dt=0.05, steps=120, m=48)
    p.simulate = "transpose"
    p.err_target, stops = pick_target(p)
    ref = oracle.run(p)
    assert [ref["used"][r] for r in range(p.o)] == stops
    got = run_gpu(ctx, p)
    check(got, ref, p, 1e-9, True)
    for r in range(p.o):
        assert abs(got["err_bound"][r] - ref["err"][r]) <= 1e-9 * max(ref["err"][r], 1e-300)


def test_transposed_through_the_server(ctx):
    p = W.random_csr_problem(5000, seed=8, n_gen=6, o=2, c_width=500, dt=0.01, steps=200, m=30)
    p.simulate = "auto"
    solo = run_gpu(ctx, p, expm_mode="propagate")
    srv = kv.Server(ctx, slots=2)
    try:
        t = srv.submit(p, expm_mode="propagate")
        out = None
        for _ in range(20000):
            out = srv.poll(t)
            if out is not None:
                break
            import time
            time.sleep(0.001)
        assert out is not None
    finally:
        srv.close()
    assert out["m_used"].shape == (2,) and np.array_equal(out["m_used"], solo["m_used"])
    assert np.array_equal(out["hi"], solo["hi"]) and np.array_equal(out["lo"], solo["lo"])


_FULL_REF = {}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_random_csr_full_size_transposed(ctx, precision):
    """The benchmark's random-CSR query at full size (n = 2e6, i = 17 with the
    fixed column, o = 2, m = 60, 2000 steps, PROPAGATE as the benchmark runs
    it) by the transpose dynamics: both runs against the oracle's."""
    p64 = W.random_csr_problem(2_000_000, seed=0)
    p64.simulate = "transpose"
    if "ref" not in _FULL_REF:
        _FULL_REF["ref"] = oracle.run(p64)
    ref = _FULL_REF["ref"]
    p = W.random_csr_problem(2_000_000, seed=0, precision=precision)
    p.simulate = "transpose"
    got = run_gpu(ctx, p, expm_mode="propagate")
    check(got, ref, p64, 1e-9 if precision == "fp64" else 1e-6, False)
