"""Pins of the oracle's a-posteriori error control (Lemma 1 of Sec. 4.2 with
the growth rule of Alg. 2 / Alg. 4) against closed forms, the paper's printed
Krylov dimensions, the true Krylov error on small systems, and eigenvalue
routines."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads as W


def trapezoid(f, dt):
    return float(np.sum(0.5 * dt * (f[1:] + f[:-1])))


def test_checkpoints_contain_the_papers_dimensions(golden_dir):
    """k = 4, then ceil(1.1 k) in double: the paper's reported dimensions 544
    (Sec. 5.3) and 5932 (Sec. 4.3, 5.3) are on this sequence; the integer
    rule ceil(11 k / 10) leaves it at 187 and reaches neither."""
    g = json.load(open(os.path.join(golden_dir, "krylov_dims.json")))
    seq = oracle.checkpoints(7000)
    assert seq[:12] == [4, 5, 6, 7, 8, 9, 10, 11, 13, 15, 17, 19]
    for d in g["dimensions"]:
        assert d["k"] in seq, d
    k, ints = 4, []
    while k < 7000:
        ints.append(k)
        k = -(-11 * k // 10)
    assert all(d["k"] not in ints for d in g["dimensions"])
    assert 188 in seq and 187 in ints       # where the two rules part
    assert oracle.checkpoints(4) == [] and oracle.checkpoints(5) == [4]


@pytest.mark.parametrize("mu", [-3.0, 0.0, 0.7])
def test_lemma1_one_dimensional(mu):
    """k = 1: h(t) = e^{alpha t}; the trapezoid sum over t_j = j dt is a
    geometric series; the factor is e^{max(mu,0) T}."""
    alpha, beta, dt, steps = -2.5, 0.3, 0.05, 40
    H = np.array([[alpha], [beta]])
    r = math.exp(alpha * dt)
    S = (1 - r ** (steps + 1)) / (1 - r)
    trap = dt * (S - 0.5 * (1 + r ** steps))
    want = beta * math.exp(max(mu, 0.0) * steps * dt) * trap
    assert oracle.lemma1(H, 1, mu, dt, steps) == pytest.approx(want, rel=1e-13)


def test_lemma1_two_by_two_picks_the_k1_entry():
    """Non-symmetric Hessenberg 2 x 2: (e^{tH})_{21} = c (e^{l1 t} - e^{l2 t}) /
    (l1 - l2), distinct from the (1,2) entry (b instead of c) and the (1,1)
    entry; h_{32} multiplies."""
    a, b, c, d, h32 = -1.0, 0.8, 0.3, -2.0, 0.45
    H = np.array([[a, b], [c, d], [0.0, h32]])
    tr, det = a + d, a * d - b * c
    disc = math.sqrt(tr * tr / 4 - det)
    l1, l2 = tr / 2 + disc, tr / 2 - disc
    dt, steps = 0.02, 150
    t = np.arange(steps + 1) * dt
    h21 = c * (np.exp(l1 * t) - np.exp(l2 * t)) / (l1 - l2)
    want = h32 * trapezoid(np.abs(h21), dt)
    got = oracle.lemma1(H, 2, -1.0, dt, steps)
    assert got == pytest.approx(want, rel=1e-12)
    h12 = b * (np.exp(l1 * t) - np.exp(l2 * t)) / (l1 - l2)
    assert abs(got - h32 * trapezoid(np.abs(h12), dt)) > 1e-3 * got


def test_lemma1_zero_subdiagonal():
    H = np.array([[-1.0, 0.2], [0.2, -3.0], [0.0, 0.0]])
    assert oracle.lemma1(H, 2, 5.0, 0.1, 10) == 0.0


def dense_of(system, n):
    return np.stack([oracle.apply(system, np.eye(n)[i]) for i in range(n)], axis=1)


def krylov_all_rows(system, v, m, method):
    """Krylov run with C = I, so P = V (n x m) and the approximation
    V_k e^{t H_k} e_1 can be formed for any k."""
    n = len(v)
    rp = np.arange(n + 1, dtype=np.int64)
    return oracle.krylov(system, v, m, rp, np.arange(n, dtype=np.int64), np.ones(n), method=method)


@pytest.mark.parametrize("case", ["heat2d", "heat3d", "nonsym"])
def test_lemma1_bounds_the_true_error(case):
    """|| e^{tA} v - V_k e^{t H_k} e_1 || <= bound for every output time and
    several k (exact exponentials by scipy on small systems; a fine output
    grid so the trapezoid integral is accurate)."""
    rng = np.random.default_rng(11)
    if case == "heat2d":
        sysm = W.GridSystem(dims=(9, 7), coef=0.01, h=(0.1, 0.125))
        method, dt, steps = "lanczos", 0.02, 200
    elif case == "heat3d":
        sysm = W.GridSystem(dims=(5, 4, 6), coef=0.01, h=(1 / 6, 1 / 5, 1 / 7))
        method, dt, steps = "lanczos", 0.01, 300
    else:
        n = 40
        A = rng.standard_normal((n, n)) / math.sqrt(n) - 1.5 * np.eye(n)
        sysm = W.dense_to_csr(A)
        method, dt, steps = "arnoldi", 0.02, 150
    n = int(sysm.n)
    A = dense_of(sysm, n)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    m = 16
    H, V, used = krylov_all_rows(sysm, v, m, method)
    mu = oracle.mu_bound(sysm, False)
    ts = np.arange(steps + 1) * dt
    for k in (3, 6, 10, 15):
        bound = oracle.lemma1(H, k, mu, dt, steps)
        worst = 0.0
        for t in ts[::10]:
            exact = sl.expm(t * A) @ v
            approx = V[:, :k] @ sl.expm(t * H[:k, :k])[:, 0]
            worst = max(worst, float(np.linalg.norm(exact - approx)))
        assert worst <= bound * (1 + 1e-6) + 1e-15, (k, worst, bound)
        assert bound > 0.0


def test_mu_grid_is_the_largest_laplacian_eigenvalue():
    """The closed form against the eigenvalues of the operator assembled
    column by column through the oracle's stencil."""
    for dims, h in [((7, 5), (0.125, 1 / 6)), ((4, 6, 3), (0.2, 1 / 7, 0.25))]:
        sysm = W.GridSystem(dims=dims, coef=0.01, h=h)
        n = int(np.prod(dims))
        lam = np.linalg.eigvalsh(dense_of(sysm, n))
        assert oracle.mu_bound(sysm, False) == pytest.approx(lam.max(), rel=1e-12)
        assert lam.max() < 0


def test_mu_csr_gershgorin():
    """Gershgorin of the symmetric part: exact for a diagonal matrix, an upper
    bound of lambda_max((A + A^T)/2) otherwise, and of the augmented matrix's
    for a column that carries the constant."""
    d = np.array([-3.0, -1.0, -2.0])
    assert oracle.mu_bound(W.dense_to_csr(np.diag(d)), False) == -1.0
    rng = np.random.default_rng(2)
    for _ in range(5):
        A = rng.standard_normal((12, 12)) * (rng.random((12, 12)) < 0.3) - 2 * np.eye(12)
        sysm = W.dense_to_csr(A)
        lam = np.linalg.eigvalsh(0.5 * (A + A.T)).max()
        g = oracle.mu_bound(sysm, False)
        assert g >= lam - 1e-12
        sysm.b = rng.uniform(-0.5, 0.5, 12)
        Aa = np.zeros((13, 13))
        Aa[:12, :12] = A
        Aa[:12, 12] = sysm.b
        lam_a = np.linalg.eigvalsh(0.5 * (Aa + Aa.T)).max()
        ga = oracle.mu_bound(sysm, True)
        assert ga >= lam_a - 1e-12 and ga >= g
        assert oracle.mu_bound(sysm, False) == g   # a generator column works on A


def test_error_control_stops_at_the_first_checkpoint_below_target():
    p = W.heat2d_20()
    p.m, p.err_target = 64, 1e-6
    r = oracle.run(p)
    k = r["used"][0]
    checks = r["checks"][0]
    assert k in oracle.checkpoints(64) and checks[-1] == (k, r["err"][0])
    assert r["err"][0] < 1e-6 and all(e >= 1e-6 for _, e in checks[:-1])
    assert [c for c, _ in checks] == oracle.checkpoints(64)[:len(checks)]
    # the first k columns of H do not depend on later iterations: the
    # fixed-m run with m = k gives the same H, bounds and error bound (up to
    # the summation order of the oracle's threaded dot products, ~1e-14)
    q = W.heat2d_20()
    q.m = k
    f = oracle.run(q)
    Hr = r["H"][0][:k + 1, :k]
    assert np.max(np.abs(f["H"][0][:k + 1, :k] - Hr)) <= 1e-12 * np.max(np.abs(Hr))
    assert np.max(np.abs(f["hi"] - r["hi"])) <= 1e-12 * np.max(np.abs(r["hi"]))
    assert f["err"][0] == pytest.approx(r["err"][0], rel=1e-9)


def test_error_control_unreachable_target_runs_to_m():
    p = W.heat2d_20()
    p.m, p.err_target = 24, 1e-12
    r = oracle.run(p)
    assert r["used"][0] == 24 and r["err"][0] >= 1e-12
    assert len(r["checks"][0]) == len(oracle.checkpoints(24))


def test_breakdown_gives_zero_bound():
    """n = 9 (3 x 3 grid): the space is exhausted before m; the bound at the
    dimension reached is (numerically) zero and no later checkpoint runs."""
    p = W.heat((3, 3), block=(1, 1), output="centre", dt=0.05, steps=40, m=30)
    p.err_target = 1e-14
    r = oracle.run(p)
    u = r["used"][0]
    assert u < 9 and r["err"][0] < 1e-10
    assert all(k < u for k, _ in r["checks"][0])
