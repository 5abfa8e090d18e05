"""Pins of the paper's 3-D heat benchmark as read here (Sec. 5.3: a unit
cube, insulated except the x = 1 face, which exchanges heat with the ambient
at constant 0.5; cell-centred finite volumes) and of the oracle on it: the
operator's structure (insulated faces conserve heat; only the x = 1 face
loses it; symmetric, negative definite), the oracle's output against the
closed form of the separable exponential, within the oracle's own Lemma-1
bound, and heat conservation when nothing is exchanged."""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import oracle
import workloads as W


def dense(sysm):
    return sp.csr_matrix((sysm.val, sysm.col, sysm.row_ptr), shape=(sysm.n, sysm.n)).toarray()


def test_operator_structure():
    N, c, kappa = 5, 0.01, 0.5
    h = 1.0 / N
    A = dense(W.paper_heat(N, steps=1, m=4).system)
    assert np.array_equal(A, A.T)
    # interior coupling coef/h^2 to each of the 6 neighbours
    mid = (2 * N + 2) * N + 2
    assert np.count_nonzero(A[mid]) == 7 and np.isclose(A[mid, mid], -6 * c / h ** 2)
    # insulated faces: no heat leaves a cell that does not touch x = 1
    x = np.arange(N ** 3) % N
    rows = A.sum(axis=1)
    assert np.allclose(rows[x < N - 1], 0.0, atol=1e-12)
    # the x = 1 face: the Robin flux through the half cell, -g/h per cell
    g = kappa * (2 * c / h) / (2 * c / h + kappa)
    assert np.allclose(rows[x == N - 1], -g / h, atol=1e-12)
    assert np.max(np.linalg.eigvalsh(A)) < 0.0


def closed_form(N, dt, steps, coef=0.01, exchange=0.5):
    """Centre temperature per unit initial temperature: e^{At} is the
    Kronecker product of the three 1-D exponentials, and both the heated
    block and the 8-cell centre average are separable."""
    factors = W.paper_heat_factors(N, coef, exchange)
    centres = (np.arange(N) + 0.5) / N
    lims = (0.4, 0.2, 0.1)
    cvec = np.zeros(N)
    cvec[[N // 2 - 1, N // 2]] = 0.5
    y = np.ones(steps + 1)
    for Ad, lim in zip(factors, lims):
        b = (centres <= lim).astype(float)
        M = sl.expm(Ad * dt)
        u = b.copy()
        for k in range(steps + 1):
            y[k] *= cvec @ u
            u = M @ u
    return y


def test_oracle_against_the_separable_closed_form():
    N, dt, steps = 16, 0.2, 100            # T = 20 as in the paper, coarser steps
    p = W.paper_heat(N, dt=dt, steps=steps, m=300, err_target=1e-10)
    r = oracle.run(p)
    y = closed_form(N, dt, steps)
    S = np.max(y)
    assert S > 1e-3                        # heat reaches the centre within T
    b0 = r["beta0"][0]
    # hi = 1.1 y, lo = 0.9 y for a non-negative y; the basis row is y itself
    assert np.max(np.abs(r["basis"][0][0] - y)) <= 1e-9 * S
    # the output error is within the Lemma-1 bound times ||C|| ||E||
    err = np.max(np.abs(r["basis"][0][0] - y))
    assert err <= b0 * np.sqrt(8 * 0.125 ** 2) * r["err"][0] + 1e-15
    assert r["used"][0] < 300
    assert np.allclose(r["hi"][0], 1.1 * np.maximum(y, 0) + 0.9 * np.minimum(y, 0), rtol=0, atol=1e-9 * S)


def test_heat_is_conserved_without_exchange():
    """exchange = 0: every face insulated, the total heat (C = all ones)
    stays at the initial heat at every step."""
    N = 8
    p = W.paper_heat(N, dt=0.5, steps=40, m=60, exchange=0.0)
    n = N ** 3
    p.C_row_ptr, p.C_col, p.C_val = np.array([0, n]), np.arange(n, dtype=np.int64), np.ones(n)
    r = oracle.run(p)
    total = p.columns[0].idx.size
    assert np.allclose(r["basis"][0][0], total, rtol=1e-12, atol=0)


def _kron_faces(dims, coef, h, face):
    """Independent dense form of the grid operator with face coefficients: a
    Kronecker sum of 1-D operators, each the insulated (Neumann) second
    difference coef/h^2 [1, -2, 1] with end rows [-1, 1], minus gamma on its
    two end points' diagonals."""
    mats = []
    for a, N in enumerate(dims):
        k = coef / h[a] ** 2
        T = np.zeros((N, N))
        for i in range(N - 1):
            T[i, i + 1] = T[i + 1, i] = k
            T[i, i] -= k
            T[i + 1, i + 1] -= k
        T[0, 0] -= face[2 * a]
        T[N - 1, N - 1] -= face[2 * a + 1]
        parts = [np.eye(dims[b]) if b != a else T for b in reversed(range(len(dims)))]
        K = parts[0]
        for q in parts[1:]:
            K = np.kron(K, q)
        mats.append(K)
    return sum(mats)


@pytest.mark.parametrize("dims", [(6, 5), (5, 4, 3), (4, 6, 7)])
def test_grid_apply_with_faces_matches_kronecker_sum(dims):
    rng = np.random.default_rng(len(dims) + dims[0])
    h = tuple(1.0 / d for d in dims)
    face = tuple(float(v) for v in rng.uniform(0.0, 3.0, 2 * len(dims)))
    sysm = W.GridSystem(dims=dims, coef=0.01, h=h, face=face)
    x = rng.standard_normal(sysm.n)
    A = _kron_faces(dims, 0.01, h, face)
    assert np.allclose(oracle.apply(sysm, x), A @ x, rtol=1e-13, atol=1e-13)


def test_grid_faces_at_the_dirichlet_value_give_the_dirichlet_operator():
    dims, coef = (7, 6, 5), 0.01
    h = tuple(1.0 / (d + 1) for d in dims)
    face = tuple(coef / h[a // 2] ** 2 for a in range(6))
    x = np.random.default_rng(3).standard_normal(7 * 6 * 5)
    a = oracle.apply(W.GridSystem(dims=dims, coef=coef, h=h, face=face), x)
    b = oracle.apply(W.GridSystem(dims=dims, coef=coef, h=h), x)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-13)


def test_paper_heat_grid_is_the_paper_heat_csr_operator():
    """The matrix-free form of the paper's heat model (insulated faces,
    exchange at x = 1) is the CSR matrix paper_heat builds from the 1-D
    factors, and the oracle's whole run on it gives the same outputs."""
    N = 10
    g = W.paper_heat_grid(N, dt=0.2, steps=50, m=40)
    c = W.paper_heat(N, dt=0.2, steps=50, m=40)
    x = np.random.default_rng(4).standard_normal(N ** 3)
    assert np.allclose(oracle.apply(g.system, x), dense(c.system) @ x, rtol=1e-13, atol=1e-13)
    assert np.array_equal(W.column_dense(g.columns[0], N ** 3, g.system.dims),
                          W.column_dense(c.columns[0], N ** 3))
    rg, rc = oracle.run(g), oracle.run(c)
    S = np.max(np.abs(rc["hi"]))
    assert np.max(np.abs(rg["hi"] - rc["hi"])) <= 1e-12 * S
    assert oracle.mu_bound(g.system, False) == 0.0
