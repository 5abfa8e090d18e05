"""Pins of the CPU oracle against facts that do not come from the oracle itself:
values printed in the paper, closed forms, library routines on special cases,
invariants and brute force.  CPU only (no GPU marker)."""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import oracle
import workloads as W


# ------------------------------------------------------------------ expm ---
@pytest.mark.parametrize("m", [1, 2, 5, 13, 30, 41])
@pytest.mark.parametrize("scale", [1e-3, 0.7, 5.0, 60.0, 900.0])
def test_expm_matches_scipy(m, scale):
    """Pade-13 with scaling and squaring against scipy's expm (an independent
    implementation of Higham 2005 / Al-Mohy-Higham 2009) over norms that need
    no scaling up to ~8 squarings."""
    rng = np.random.default_rng(m * 1000 + int(scale * 10))
    A = rng.standard_normal((m, m))
    A *= scale / max(np.linalg.norm(A, 1), 1e-300)
    # stable-ish spectrum for large norms, so exp(A) stays representable
    if scale > 10:
        A -= (scale * 0.6) * np.eye(m)
    E = oracle.expm(A)
    R = scipy.linalg.expm(A)
    err = np.linalg.norm(E - R, 1) / max(np.linalg.norm(R, 1), 1e-300)
    assert err < 2e-12 * max(1.0, scale / 5.0), err


def test_expm_closed_forms():
    """Special cases whose exponential is known exactly."""
    d = np.array([-3.0, -0.5, 0.0, 0.25, 2.0])
    assert np.allclose(oracle.expm(np.diag(d)), np.diag(np.exp(d)), rtol=1e-14, atol=0)
    for t in [0.1, math.pi / 4, 3 * math.pi / 4, 7.3, 40.0]:
        R = oracle.expm(np.array([[0.0, t], [-t, 0.0]]))
        ref = np.array([[math.cos(t), math.sin(t)], [-math.sin(t), math.cos(t)]])
        assert np.max(np.abs(R - ref)) < 1e-13 * max(1.0, t)
    # nilpotent Jordan block: exp(tN) = sum_k t^k N^k / k!
    N = np.diag(np.ones(4), 1)
    t = 2.5
    ref = sum(np.linalg.matrix_power(N * t, k) / math.factorial(k) for k in range(5))
    assert np.max(np.abs(oracle.expm(N * t) - ref)) < 1e-13 * np.max(np.abs(ref))
    assert np.array_equal(oracle.expm(np.zeros((3, 3))), np.eye(3))


def test_pade13_normalised_coefficients():
    """b_0 and b_1 of the degree-13 Pade approximant (Higham 2005 Table 10.4),
    seen through exp of a 1x1 matrix: r(x) = p(x)/p(-x), and exp(1x1) must
    agree with math.exp over the unscaled range; for x < 0 the even and odd
    parts cancel, so the relative error grows like e^{|x|} u."""
    for x in [-5.3, -1.0, -1e-8, 0.0, 1e-8, 0.5, 5.3]:
        tol = 4e-16 * math.exp(abs(x))
        assert abs(oracle.expm(np.array([[x]]))[0, 0] - math.exp(x)) <= tol * math.exp(x)


# ----------------------------------------------------------------- A x ---
def _kron_laplacian(dims, coef, h):
    """Independent construction: sum over axes of I (x) T_axis (x) I / h^2."""
    mats = []
    for a, n in enumerate(dims):
        T = sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / h[a] ** 2
        # flat index (z*ny + y)*nx + x: kron order is z, y, x (x fastest)
        parts = [sp.identity(dims[b]) if b != a else T for b in reversed(range(len(dims)))]
        K = parts[0]
        for p in parts[1:]:
            K = sp.kron(K, p)
        mats.append(K)
    return coef * sum(mats)


@pytest.mark.parametrize("dims", [(7,), (5, 4), (6, 3, 4), (20, 20)])
def test_grid_apply_matches_kronecker_sum(dims):
    if len(dims) == 1:
        dims = (dims[0], 1)
    h = tuple(1.0 / (d + 1) for d in dims)
    sysm = W.GridSystem(dims=dims, coef=0.01, h=h)
    x = np.random.default_rng(1).standard_normal(sysm.n)
    L = _kron_laplacian(dims, 0.01, h)
    assert np.allclose(oracle.apply(sysm, x), L @ x, rtol=1e-13, atol=1e-12)


def test_csr_apply_augmented():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((9, 9)) * (rng.random((9, 9)) < 0.4)
    b = rng.standard_normal(9)
    sysm = W.dense_to_csr(A, b=b)
    x = rng.standard_normal(10)
    Aa = np.zeros((10, 10))
    Aa[:9, :9] = A
    Aa[:9, 9] = b
    assert np.allclose(oracle.apply(sysm, x, aug=True), Aa @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(oracle.apply(sysm, x[:9]), A @ x[:9], rtol=1e-14, atol=1e-14)


def test_heat_norm_reading():
    """||A t|| at t = 50 on the 100^3 grid is printed as 32,771,611 (Sec. 4.2).
    With coefficient 0.01 on the Laplacian with h = 1/101 and the Frobenius
    norm (closed form: 7 entries per interior row) the Dirichlet grid gives a
    value within 1% of it; the paper's insulated/Robin boundary differs only on
    boundary rows.  This pins the reading 'diffusivity 0.01 multiplies L/h^2'
    (alpha^2 = 1e-4 would be 100x off)."""
    N, h, t = 100, 1.0 / 101, 50.0
    k = 0.01 / h ** 2
    # per axis: N-1 off-diagonal pairs per line, N^2 lines, 2 entries each
    off = 3 * 2 * (N - 1) * N * N
    fro = t * k * math.sqrt(N ** 3 * 36 + off)
    assert abs(fro / 32771611 - 1) < 0.01


# ----------------------------------------------------- worked example -----
def test_oscillator_paper_values(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "oscillator.json")))
    p = W.oscillator()
    r = oracle.run(p)
    tol = g["printed_digits_tol"]
    k = g["violation_step"]
    # basis matrix C e^{At} E at 3 pi / 4 (Fig. 2(c))
    assert abs(r["basis"][0][0, k] - g["basis_at_violation"]["i_y"]) < tol
    assert abs(r["basis"][1][0, k] - g["basis_at_violation"]["i_f"]) < tol
    assert r["viol_step"] == k and r["viol_row"] == 0
    for s in g["no_violation_steps"]:
        assert r["hi"][0, s] < p.theta[0]
    # the paper's LP point reaches x = 4 (equality) with y0 = 0.66: check our
    # basis maps it there, and its y(t) and t agree with the printed state
    x0 = g["lp_initial_point"]
    x_at = r["basis"][1][0, k] * 1.0 + r["basis"][0][0, k] * x0[1]
    assert abs(x_at - g["lp_final_point"][0]) < tol
    # y component: project with C = (0, 1, 0)
    py = W.oscillator()
    py.C_col = np.array([1], dtype=np.int64)
    ry = oracle.run(py)
    y_at = ry["basis"][1][0, k] + ry["basis"][0][0, k] * x0[1]
    assert abs(y_at - g["lp_final_point"][1]) < tol
    # t component: C = (0, 0, 1), the affine term integrates to t
    pt = W.oscillator()
    pt.C_col = np.array([2], dtype=np.int64)
    rt = oracle.run(pt)
    assert abs(rt["basis"][1][0, k] - g["lp_final_point"][2]) < tol
    # full-state basis rows (Fig. 2(a)) from unit initial vectors
    for row, key in [(0, "basis_full_at_violation_row_x"), (1, "basis_full_at_violation_row_y")]:
        for jcol in range(2):
            e = np.zeros(3)
            e[jcol] = 1.0
            q = W.oscillator()
            q.columns = [W.Column(kind="dense", zlo=0, zhi=1, dense=e)]
            q.C_col = np.array([row], dtype=np.int64)
            rq = oracle.run(q)
            assert abs(rq["basis"][0][0, k] - g[key][jcol]) < tol
    # happy breakdowns (Sec. 4.2: the loop stops early and is exact)
    assert r["used"][1] == g["krylov_dim_fixed_column"]
    assert r["used"][0] == g["krylov_dim_generator"]


def test_oscillator_exact_closed_form():
    """x(t) = -5 cos t + y0 sin t: interval over y0 in [0, 1] at every step."""
    p = W.oscillator()
    r = oracle.run(p)
    for k in range(p.steps + 1):
        t = k * p.dt
        vals = [-5 * math.cos(t) + y0 * math.sin(t) for y0 in (0.0, 1.0)]
        assert abs(r["lo"][0, k] - min(vals)) < 1e-12
        assert abs(r["hi"][0, k] - max(vals)) < 1e-12
    assert np.allclose(r["zstar"], [1.0, 1.0])
    assert abs(r["ystar"] - (5 / math.sqrt(2) + 1 / math.sqrt(2))) < 1e-12


# ----------------------------------------------- full-dimension Krylov ----
def _dense_reference_basis(A, b, cols, Crows, dt, steps):
    """C e^{A' t} E_j with scipy's dense expm of the augmented matrix."""
    n = A.shape[0]
    aug = b is not None
    N = n + (1 if aug else 0)
    Aa = np.zeros((N, N))
    Aa[:n, :n] = A
    if aug:
        Aa[:n, n] = b
    out = []
    for vec in cols:
        res = np.zeros((Crows.shape[0], steps + 1))
        for k in range(steps + 1):
            x = scipy.linalg.expm(Aa * (k * dt)) @ vec
            res[:, k] = Crows @ x[:n]
        out.append(res)
    return out


@pytest.mark.parametrize("method", ["arnoldi", "lanczos"])
@pytest.mark.parametrize("n", [6, 17])
def test_krylov_full_dimension_is_exact(method, n):
    """With m = n the Krylov approximation is exact (or breaks down earlier
    with the invariant subspace), so the basis must equal C e^{At} E_j."""
    rng = np.random.default_rng(n)
    if method == "lanczos":
        sysm = W.random_symmetric_csr(n, seed=n)
        A = np.zeros((n, n))
        for r in range(n):
            for e in range(sysm.row_ptr[r], sysm.row_ptr[r + 1]):
                A[r, sysm.col[e]] = sysm.val[e]
        b = None
    else:
        A = rng.standard_normal((n, n)) * 0.6 - 0.8 * np.eye(n)
        b = rng.standard_normal(n) * 0.3
        sysm = W.dense_to_csr(A, b=b)
    p = W.random_problem(sysm, seed=n, n_cols=3, o=2, dt=0.15, steps=12, m=n + (1 if b is not None else 0),
                         fixed_last=b is not None, method=method)
    r = oracle.run(p)
    Crows = np.zeros((p.o, n))
    for rr in range(p.o):
        for e in range(p.C_row_ptr[rr], p.C_row_ptr[rr + 1]):
            Crows[rr, p.C_col[e]] += p.C_val[e]
    vecs = []
    for c in p.columns:
        v = c.dense.copy()
        if b is not None:
            v = np.concatenate([v, [1.0 if c.is_fixed else 0.0]])
        vecs.append(v)
    ref = _dense_reference_basis(A, b, vecs, Crows, p.dt, p.steps)
    for j in range(p.i):
        S = np.max(np.abs(ref[j]))
        assert np.max(np.abs(r["basis"][j] - ref[j])) <= 1e-10 * S


def test_lanczos_and_arnoldi_agree_on_symmetric():
    sysm = W.random_symmetric_csr(60, seed=3)
    p = W.random_problem(sysm, seed=5, n_cols=2, o=2, m=15, steps=20, dt=0.1)
    pl = W.random_problem(sysm, seed=5, n_cols=2, o=2, m=15, steps=20, dt=0.1, method="lanczos")
    pa = W.random_problem(sysm, seed=5, n_cols=2, o=2, m=15, steps=20, dt=0.1, method="arnoldi")
    rl, ra = oracle.run(pl), oracle.run(pa)
    for j in range(p.i):
        Hl, Ha = rl["H"][j], ra["H"][j]
        assert np.max(np.abs(Hl - Ha)) < 1e-10 * np.max(np.abs(Ha))
        assert np.max(np.abs(rl["basis"][j] - ra["basis"][j])) < 1e-10 * np.max(np.abs(ra["basis"][j]))


# ------------------------------------------------------- heat closed form -
def _heat_factor(N, coef, t, b_hi, cells):
    """1-D factor (e^{coef/h^2 T_N t} 1_[0,b_hi))[cells] by the sine eigenbasis
    of the Dirichlet second-difference matrix T_N (DST-I)."""
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)
    lam = -4.0 * np.sin(j * np.pi / (2 * (N + 1))) ** 2 * coef / h ** 2
    i = np.arange(1, N + 1)
    Q = np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(i, j) * np.pi / (N + 1))
    u0 = np.zeros(N)
    u0[:b_hi] = 1.0
    coeff = Q.T @ u0
    vals = Q[np.asarray(cells)] @ (np.exp(lam * t) * coeff)
    return vals


def _heat_closed_form(p):
    s = p.system
    N = s.dims[0]
    assert all(d == N for d in s.dims)
    b_hi = p.columns[0].box_hi[0]
    # recover the output cells from C (x fastest)
    idx = p.C_col
    coords = []
    for q in idx:
        c = []
        for _ in s.dims:
            c.append(int(q % N))
            q //= N
        coords.append(c)
    per_axis = sorted(set(c[0] for c in coords))
    out = np.zeros(p.steps + 1)
    for k in range(p.steps + 1):
        t = k * p.dt
        f = _heat_factor(N, s.coef, t, b_hi, per_axis)
        # separable: mean over the product of per-axis cells
        out[k] = np.mean(f) ** len(s.dims)
    return out


@pytest.mark.parametrize("shape,m,block,steps,dt,output", [
    ((20, 20), 80, (5, 5), 500, 0.1, "centre"),        # 2D cfg shape with adequate m
    ((12, 12, 12), 90, (3, 3, 3), 200, 0.02, "centre8"),
])
def test_heat_lanczos_matches_closed_form(shape, m, block, steps, dt, output):
    p = W.heat(shape, block=block, output=output, dt=dt, steps=steps, m=m)
    r = oracle.run(p)
    ref = _heat_closed_form(p)
    S = np.max(np.abs(ref))
    assert S > 0
    assert np.max(np.abs(r["basis"][0][0] - ref)) <= 1e-9 * S
    # maximum principle at adequate m: 0 <= lo <= hi <= 1.1
    assert r["lo"].min() >= -1e-9 * S and r["hi"].max() <= 1.1 + 1e-9


def test_heat_small_m_exact_zero_beyond_reach():
    """v_j is supported within j-1 stencil hops of the heated block, so an
    output cell further away than m-1 hops sees exactly 0 (cfg 100^3/m=40 has
    the centre 120 hops out)."""
    p = W.heat((30, 30, 30), block=(3, 3, 3), output="centre", dt=0.02, steps=50, m=30)
    # hop distance from block corner (2,2,2) to (15,15,15) is 39 > m - 1
    r = oracle.run(p)
    assert np.all(r["P"][0] == 0.0)
    assert np.all(r["hi"] == 0.0) and np.all(r["lo"] == 0.0)
    p2 = W.heat((30, 30, 30), block=(3, 3, 3), output="centre", dt=0.02, steps=50, m=45)
    r2 = oracle.run(p2)
    assert np.any(r2["P"][0] != 0.0)


def test_truncated_grid_reproduces_full_grid_coefficients():
    """The support argument behind the 1000^3 parity test: the same h on a
    truncated grid gives the same Lanczos coefficients while the Krylov vectors
    cannot reach the cut (checked here on 40^3 vs 16^3, block 4, m = 10)."""
    full = W.heat((40, 40, 40), block=(4, 4, 4), output="centre", dt=0.02, steps=10, m=10)
    tr = W.heat3d_truncated(full, 16)
    rf, rt = oracle.run(full), oracle.run(tr)
    Hf, Ht = rf["H"][0], rt["H"][0]
    assert np.max(np.abs(Hf - Ht)) <= 1e-12 * np.max(np.abs(Hf))


def test_norm_nonincreasing_symmetric_negative_definite():
    """||e^{At} v|| is non-increasing for symmetric negative-definite A; with
    C = I and full Krylov dimension the basis column is e^{At} v itself."""
    n = 25
    sysm = W.random_symmetric_csr(n, seed=11)
    rng = np.random.default_rng(4)
    rp, cc, cv = W._c_rows([([r], [1.0]) for r in range(n)])
    col = W.Column(kind="dense", zlo=0, zhi=1, dense=rng.standard_normal(n))
    p = W.Problem(system=sysm, columns=[col], C_row_ptr=rp, C_col=cc, C_val=cv,
                  theta=np.full(n, np.inf), dt=0.05, steps=60, m=n, method="lanczos")
    r = oracle.run(p)
    norms = np.linalg.norm(r["basis"][0], axis=0)
    assert np.all(np.diff(norms) <= 1e-12 * norms[0])
    assert abs(norms[0] - np.linalg.norm(col.dense)) < 1e-12 * norms[0]


# ----------------------------------------------------------- bounds -------
@pytest.mark.parametrize("seed", range(6))
def test_bounds_match_vertex_enumeration(seed):
    """The closed-form interval equals min/max over all 2^i box vertices; the
    first violation and the counter-example vertex agree with brute force."""
    rng = np.random.default_rng(seed)
    ncol, o, S = 4, 3, 9
    basis = rng.standard_normal((ncol, o, S))
    basis[1, :, 2] = 0.0                       # exercise p == 0
    zlo = -rng.random(ncol)
    zhi = rng.random(ncol)
    zlo[3] = zhi[3] = 1.0                       # a fixed column
    theta = np.array([1.5, 0.8, 2.0]) + 0.3 * seed
    r = oracle.bounds(basis, zlo, zhi, theta)
    verts = np.array(list(itertools.product(*[(zlo[j], zhi[j]) for j in range(ncol)])))
    first = None
    for k in range(S):
        for rr in range(o):
            vals = verts @ basis[:, rr, k]
            assert abs(r["lo"][rr, k] - vals.min()) < 1e-12
            assert abs(r["hi"][rr, k] - vals.max()) < 1e-12
            if first is None and vals.max() >= theta[rr]:
                first = (k, rr)
    if first is None:
        assert r["viol_step"] == -1
    else:
        assert (r["viol_step"], r["viol_row"]) == first
        k, rr = first
        y = float(np.dot(r["zstar"], basis[:, rr, k]))
        assert abs(y - r["ystar"]) < 1e-12 and y >= theta[rr]
        assert np.all(r["zstar"] >= zlo - 1e-15) and np.all(r["zstar"] <= zhi + 1e-15)


def test_arnoldi_output_matches_expm_multiply_on_random_csr():
    """The random-CSR workload shape (n = 2e4, 16 unit generators + the fixed
    column carrying the constant, m = 60): the oracle's projected Arnoldi output
    C V e^{H t} e_1 beta0 equals C e^{A' t} E_j from scipy's expm_multiply
    (Al-Mohy & Higham 2011) although modified Gram-Schmidt loses orthogonality
    on this non-normal A -- the Arnoldi relation still holds."""
    import scipy.sparse.linalg as spl
    p = W.random_csr_problem(20000, seed=0, m=60, steps=40, dt=0.05)
    s = p.system
    n = s.n
    A = sp.csr_matrix((s.val, s.col, s.row_ptr), shape=(n, n))
    Aa = sp.bmat([[A, sp.csr_matrix(s.b.reshape(-1, 1))], [sp.csr_matrix((1, n)), sp.csr_matrix((1, 1))]]).tocsr()
    Crows = np.zeros((p.o, n + 1))
    for r in range(p.o):
        Crows[r, p.C_col[p.C_row_ptr[r]:p.C_row_ptr[r + 1]]] = p.C_val[p.C_row_ptr[r]:p.C_row_ptr[r + 1]]
    r = oracle.run(p, columns=[0, 16])
    for j in (0, 16):
        c = p.columns[j]
        e = np.concatenate([W.column_dense(c, n), [1.0 if c.is_fixed else 0.0]])
        X = spl.expm_multiply(Aa, e, start=0.0, stop=p.steps * p.dt, num=p.steps + 1, endpoint=True)
        ref = (Crows @ X.T)
        S = np.max(np.abs(ref))
        assert np.max(np.abs(r["basis"][j] - ref)) <= 1e-10 * S
