"""Pins of the oracle's transpose-dynamics simulation (Sec. 4.1: the basis
matrix C e^{At} E from o simulations of x' = A^T x started at the rows of C
and projected by E^T) against the paper's worked example, dense transposes,
and the forward simulation where both are exact."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads as W


def dense_augmented(sysm):
    n = int(sysm.n)
    A = np.zeros((n + 1, n + 1))
    for r in range(n):
        for e in range(sysm.row_ptr[r], sysm.row_ptr[r + 1]):
            A[r, sysm.col[e]] = sysm.val[e]
    if sysm.b is not None:
        A[:n, n] = sysm.b
    return A


def test_transpose_apply_is_the_dense_transpose():
    rng = np.random.default_rng(4)
    sysm = W.random_csr(50, nnz_per_row=5, seed=3)
    Aa = dense_augmented(sysm)
    x = rng.standard_normal(51)
    assert np.allclose(oracle.apply(sysm, x, aug=True, trans=True), Aa.T @ x, rtol=0, atol=1e-13)
    assert np.allclose(oracle.apply(sysm, x[:50], trans=True), Aa[:50, :50].T @ x[:50], rtol=0, atol=1e-13)
    g = W.GridSystem(dims=(5, 4), coef=0.01, h=(1 / 6, 0.2))
    y = rng.standard_normal(20)
    assert np.array_equal(oracle.apply(g, y, trans=True), oracle.apply(g, y))  # symmetric


def test_oscillator_transpose_worked_example(golden_dir):
    """Sec. 4.1: one simulation of the transpose dynamics from the output
    direction (1, 0, 0, 0) reaches (-0.707, 0.707, 0, 0) at 3 pi / 4, whose
    projection by E^T is the basis row (0.707, 3.54); the violation is at
    step 3 as in the forward computation."""
    g = json.load(open(os.path.join(golden_dir, "oscillator.json")))
    tol = g["printed_digits_tol"]
    p = W.oscillator()
    n = p.system.n
    # the state: C = I projection, so P = V and V e^{H t} e_1 is the state
    H, V, u = oracle.krylov(p.system, np.array([1.0, 0, 0, 0]), 4, np.arange(5, dtype=np.int64),
                            np.arange(4, dtype=np.int64), np.ones(4), method="arnoldi", aug=True, trans=True)
    t = 3 * math.pi / 4
    state = V[:, :u] @ sl.expm(t * H[:u, :u])[:, 0]
    assert np.max(np.abs(state - np.array(g["transpose_state_at_violation"]))) < tol
    p.simulate = "transpose"
    r = oracle.run(p)
    assert r["transposed"] and list(r["used"].keys()) == [0]   # one run (o = 1)
    k = g["violation_step"]
    assert abs(r["basis"][0][0, k] - g["basis_at_violation"]["i_y"]) < tol
    assert abs(r["basis"][1][0, k] - g["basis_at_violation"]["i_f"]) < tol
    assert r["viol_step"] == k
    f = oracle.run(W.oscillator())
    assert np.max(np.abs(r["hi"] - f["hi"])) < 1e-12 and np.max(np.abs(r["lo"] - f["lo"])) < 1e-12


@pytest.mark.parametrize("case", ["csr_forcing", "csr_symmetric", "grid"])
def test_transpose_equals_forward_at_full_dimension(case):
    """With the Krylov dimension equal to the state dimension both sides are
    exact, so the two ways of building the basis agree (to rounding)."""
    if case == "csr_forcing":
        sysm = W.random_csr(24, nnz_per_row=4, seed=5)
        p = W.random_problem(sysm, seed=6, n_cols=4, o=2, dt=0.05, steps=30, m=25, fixed_last=True)
    elif case == "csr_symmetric":
        p = W.random_problem(W.random_symmetric_csr(30, seed=7), seed=8, n_cols=5, o=2, dt=0.05, steps=30, m=30)
    else:
        p = W.heat((5, 4, 3), block=(2, 2, 2), output="centre8", dt=0.05, steps=30, m=60)
        p.columns.append(W.Column(kind="dense", zlo=-1.0, zhi=1.0,
                                  dense=np.random.default_rng(9).standard_normal(60)))
    f = oracle.run(p)
    p.simulate = "transpose"
    t = oracle.run(p)
    S = max(np.max(np.abs(f["basis"][j])) for j in range(p.i))
    for j in range(p.i):
        assert np.max(np.abs(t["basis"][j] - f["basis"][j])) <= 1e-10 * S, j
    assert np.max(np.abs(t["hi"] - f["hi"])) <= 1e-10 * S


def test_auto_takes_the_smaller_side():
    p = W.random_csr_problem(300, seed=1, n_gen=5, o=2, c_width=50, steps=5, m=8)
    p.simulate = "auto"
    assert oracle.transposed(p)                    # o = 2 < i = 6
    q = W.heat2d_20()
    q.simulate = "auto"
    assert not oracle.transposed(q)                # i = o = 1: forward


def test_transpose_equals_forward_on_the_random_csr_workload():
    """The random-CSR workload at n = 2e4 (16 generators + the fixed column
    carrying the constant, o = 2, m = 60): 2 runs on A'^T and 17 on A' give
    the same basis, both being converged at this m (the forward side is
    itself pinned to scipy's expm_multiply)."""
    f = oracle.run(W.random_csr_problem(20000, seed=0, m=60, steps=200))
    p = W.random_csr_problem(20000, seed=0, m=60, steps=200)
    p.simulate = "transpose"
    t = oracle.run(p)
    S = max(np.max(np.abs(f["basis"][j])) for j in range(p.i))
    assert max(np.max(np.abs(t["basis"][j] - f["basis"][j])) for j in range(p.i)) <= 1e-11 * S


def test_transpose_equals_forward_on_replicated_blocks():
    """The replicated-block shape (Sec. 5.2, h = 20: n = 560, i = 160, o = 1):
    one transposed run gives the basis of the 160 forward runs (both exact:
    the Krylov spaces are invariant within 28 dimensions)."""
    t = oracle.run(W.replicated_blocks(20, simulate="transpose"))
    f = oracle.run(W.replicated_blocks(20, simulate="forward"))
    assert list(t["used"].values()) == [28] and set(f["used"].values()) == {28}
    S = max(np.max(np.abs(f["basis"][j])) for j in range(160))
    assert max(np.max(np.abs(t["basis"][j] - f["basis"][j])) for j in range(160)) <= 1e-12 * S
