"""Parity of the device per-step LP (kv_check_polytope: polyhedral unsafe
and initial sets, Sec. 2.1 over the basis of Sec. 3.1-3.2) against the
oracle's LP on the oracle's basis: margins t*_k within 1e-9 (FP64) / 1e-6
(FP32 storage) of their scale, the same first violation, and a valid
minimiser (unique only in special cases, where it is compared too)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import polytope as LP

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


def gpu_lp(ctx, p, U, v, Iz=None, iota=None, tol=0.0, **kw):
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p, **kw)
    try:
        r = ph.run()
        return r, ph.check_polytope(U, v, Iz, iota, tol)
    finally:
        ph.close()
        sysh.close()


def oracle_lp(p, U, v, Iz=None, iota=None, tol=0.0):
    r = oracle.run(p)
    B = np.stack([r["basis"][j] for j in range(p.i)])
    zlo = np.array([c.zlo for c in p.columns])
    zhi = np.array([c.zhi for c in p.columns])
    return B, zlo, zhi, LP.check(B, zlo, zhi, U, v, Iz, iota, tol)


def compare(got, ref, tol_rel, B, zlo, zhi, U, v, Iz, iota):
    assert np.array_equal(got["status"], ref["status"])
    ok = ref["status"] == LP.OPTIMAL
    scale = max(float(np.max(np.abs(ref["margin"][ok]))), 1e-300)
    err = float(np.max(np.abs(got["margin"][ok] - ref["margin"][ok]))) / scale
    assert err <= tol_rel, err
    # every minimiser is in the initial set and meets the unsafe rows relaxed by its margin
    nr = np.linalg.norm(U, axis=1)
    for k in np.nonzero(ok)[0]:
        assert LP.feasible(B[:, :, k].T, zlo, zhi, U, v + got["margin"][k] * nr, Iz, iota, got["z"][k],
                           1e-7 * max(1.0, scale)), k
    return err, scale


def oscillator_full_state():
    p = W.oscillator()
    p.C_row_ptr, p.C_col, p.C_val = W._c_rows([([0], [1.0]), ([1], [1.0]), ([2], [1.0])])
    p.theta = np.full(3, np.inf)
    return p


def test_oscillator_lp_worked_example(ctx, golden_dir):
    """Sec. 2.2: the unsafe set x = 4 is reached at 3 pi / 4 from
    (x0, y0) = (-5, 0.66), at the state (4, 3.07, 2.36)."""
    g = json.load(open(os.path.join(golden_dir, "oscillator.json")))
    p = oscillator_full_state()
    U = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    v = np.array([4.0, -4.0])
    _, got = gpu_lp(ctx, p, U, v, tol=1e-9)
    B, zlo, zhi, ref = oracle_lp(p, U, v, tol=1e-9)
    compare(got, ref, 1e-9, B, zlo, zhi, U, v, None, None)
    assert got["viol_step"] == ref["viol_step"] == g["violation_step"]
    t = g["printed_digits_tol"]
    assert abs(got["z_star"][0] - g["lp_initial_point"][1]) < t and got["z_star"][1] == pytest.approx(1.0, abs=1e-12)
    assert np.max(np.abs(got["y_star"] - np.array(g["lp_final_point"][:3]))) < t
    assert abs(got["z_star"][0] - ref["z_star"][0]) < 1e-9   # unique here (an equality)


def polygon_case(n, precision, seed=0, steps=400):
    """The random-CSR workload shape (16 generators + the fixed column, o = 2)
    with an unsafe triangle in the output plane and a budget on the
    generators (sum z_j <= 4 of the 16 in [-1, 1])."""
    p = W.random_csr_problem(n, seed=seed, m=40, steps=steps, precision=precision)
    p.theta = np.full(p.o, np.inf)
    Iz = np.zeros((1, p.i))
    Iz[0, :16] = 1.0
    iota = np.array([4.0])
    return p, Iz, iota


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_random_csr_polygon(ctx, precision):
    p64, Iz, iota = polygon_case(20000, "fp64")
    r64 = oracle.run(p64)
    B = np.stack([r64["basis"][j] for j in range(p64.i)])
    # triangle y1 >= a, y2 >= b, y1 + y2 <= c with a, b at 40% of the outputs' peak upper bounds
    hi = oracle.bounds(B, [c.zlo for c in p64.columns], [c.zhi for c in p64.columns], np.full(2, np.inf))["hi"]
    a, b = 0.4 * np.max(hi[0]), 0.4 * np.max(hi[1])
    U = np.array([[-1.0, 0.0], [0.0, -1.0], [1.0, 1.0]])
    v = np.array([-a, -b, 3.0 * (abs(a) + abs(b))])
    zlo = np.array([c.zlo for c in p64.columns])
    zhi = np.array([c.zhi for c in p64.columns])
    ref = LP.check(B, zlo, zhi, U, v, Iz, iota, 0.0)
    p, _, _ = polygon_case(20000, precision)
    _, got = gpu_lp(ctx, p, U, v, Iz, iota, 0.0, expm_mode="propagate")
    tol = 1e-9 if precision == "fp64" else 1e-6
    err, scale = compare(got, ref, tol, B, zlo, zhi, U, v, Iz, iota)
    k = ref["viol_step"]
    assert k > 0, "the case should violate"
    if abs(ref["margin"][k]) > 10 * tol * scale and abs(ref["margin"][k - 1]) > 10 * tol * scale:
        assert got["viol_step"] == k


def test_one_halfspace_equals_the_interval_bound(ctx):
    """With one unsafe row y_r >= theta the margin is theta - hi_r(k) from the
    library's own closed-form bounds (two different device paths)."""
    p = W.random_csr_problem(5000, seed=3, n_gen=6, o=3, c_width=200, dt=0.01, steps=300, m=30)
    p.theta = np.full(p.o, np.inf)
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p)
    try:
        r = ph.run()
        for row in range(p.o):
            e = np.zeros(p.o)
            e[row] = -1.0
            th = 0.3 * np.max(r["hi"][row])
            lp = ph.check_polytope(e[None, :], [-th])
            scale = np.max(np.abs(r["hi"][row])) + abs(th)
            assert np.max(np.abs(lp["margin"] - (th - r["hi"][row]))) <= 1e-12 * scale
    finally:
        ph.close()
        sysh.close()


def test_empty_initial_set(ctx):
    p = W.random_csr_problem(3000, seed=4, n_gen=3, o=2, c_width=100, dt=0.01, steps=50, m=12)
    Iz = np.zeros((1, p.i))
    Iz[0, :3] = 1.0
    _, got = gpu_lp(ctx, p, np.array([[1.0, 0.0]]), [0.0], Iz, [-3.5])   # sum of three z in [-1, 1] <= -3.5
    assert np.all(got["status"] == kv.KV_LP_EMPTY) and got["viol_step"] == -1


def test_wide_lp_many_steps(ctx):
    """40 columns (i + 1 = 41 LP rows), 5 unsafe rows, 2 initial rows, 601
    steps (one CTA each)."""
    p = W.random_csr_problem(3000, seed=5, n_gen=39, o=3, c_width=300, dt=0.01, steps=600, m=20)
    p.theta = np.full(p.o, np.inf)
    rng = np.random.default_rng(6)
    U = rng.standard_normal((5, p.o))
    v = rng.standard_normal(5) * 0.1
    Iz = rng.standard_normal((2, p.i))
    iota = np.abs(rng.standard_normal(2)) + 0.5
    _, got = gpu_lp(ctx, p, U, v, Iz, iota)
    B, zlo, zhi, ref = oracle_lp(p, U, v, Iz, iota)
    compare(got, ref, 1e-9, B, zlo, zhi, U, v, Iz, iota)


def test_lp_after_the_transpose_dynamics(ctx):
    p, Iz, iota = polygon_case(5000, "fp64", seed=7, steps=200)
    p.simulate = "transpose"
    U = np.array([[-1.0, 0.0], [0.0, -1.0]])
    v = np.array([-1e-4, -1e-4])
    _, got = gpu_lp(ctx, p, U, v, Iz, iota)
    B, zlo, zhi, ref = oracle_lp(p, U, v, Iz, iota)
    compare(got, ref, 1e-9, B, zlo, zhi, U, v, Iz, iota)


def test_lp_argument_errors(ctx):
    p = W.random_csr_problem(2000, seed=8, n_gen=2, o=2, c_width=50, dt=0.01, steps=10, m=8)
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p)
    try:
        with pytest.raises(kv.KvError) as ei:          # not run yet
            ph.check_polytope(np.array([[1.0, 0.0]]), [0.0])
        assert ei.value.code == kv.KV_EINVAL
        ph.run()
        with pytest.raises(kv.KvError) as ei:          # zero unsafe row
            ph.check_polytope(np.array([[0.0, 0.0]]), [0.0])
        assert ei.value.code == kv.KV_EINVAL
        with pytest.raises(kv.KvError) as ei:          # beyond one CTA's shared memory
            ph.check_polytope(np.ones((8000, 2)), np.ones(8000))
        assert ei.value.code == kv.KV_EINVAL
    finally:
        ph.close()
        sysh.close()


_FULL = {}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_random_csr_full_size_polygon(ctx, precision):
    """The benchmark's LP leg at full size: the random-CSR query (n = 2e6,
    i = 17, o = 2, m = 60, 2001 steps, PROPAGATE) with the unsafe triangle
    and the generator budget; margins at every 40th step against the
    oracle's LP on the oracle's basis (built by the transpose dynamics, two
    runs, which the transpose pins tie to the forward basis)."""
    if "ref" not in _FULL:
        p64 = W.random_csr_problem(2_000_000, seed=0)
        p64.simulate = "transpose"
        r = oracle.run(p64)
        B = np.stack([r["basis"][j] for j in range(p64.i)])
        zlo = np.array([c.zlo for c in p64.columns])
        zhi = np.array([c.zhi for c in p64.columns])
        hi = oracle.bounds(B, zlo, zhi, np.full(2, np.inf))["hi"]
        a, b = 0.4 * np.max(hi[0]), 0.4 * np.max(hi[1])
        U = np.array([[-1.0, 0.0], [0.0, -1.0], [1.0, 1.0]])
        v = np.array([-a, -b, 3.0 * (abs(a) + abs(b))])
        Iz = np.zeros((1, p64.i))
        Iz[0, :16] = 1.0
        iota = np.array([4.0])
        ks = np.arange(0, p64.steps + 1, 40)
        ref = np.array([LP.step_lp(B[:, :, k].T, zlo, zhi, U, v, Iz, iota)[1] for k in ks])
        _FULL["ref"] = (U, v, Iz, iota, ks, ref)
    U, v, Iz, iota, ks, ref = _FULL["ref"]
    p = W.random_csr_problem(2_000_000, seed=0, precision=precision)
    _, got = gpu_lp(ctx, p, U, v, Iz, iota, expm_mode="propagate")
    assert np.all(got["status"] == kv.KV_LP_OPTIMAL)
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got["margin"][ks] - ref)) / scale
    assert err <= (1e-6 if precision == "fp32" else 1e-9), err


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_grid_multi_column_polygon(ctx, precision):
    """A grid (Lanczos) with a point source, a dense field and a box column and
    two outputs, one of them the point cell itself; the early steps' basis
    entries of the far columns are tiny (the ill-conditioned regime of the
    LP).  Unsafe: a wedge in the output plane; initial rows: a budget on the
    first two columns.  FP32 storage feeds the LP a basis within 1e-6."""
    import math
    dims = (24, 17, 9)
    n = 24 * 17 * 9
    rng = np.random.default_rng(3)
    sysm = W.GridSystem(dims=dims, coef=0.01, h=tuple(1.0 / (d + 1) for d in dims))
    src = W.grid_index(dims, (6, 6, 4))
    cols = [W.Column(kind="sparse", zlo=-1.0, zhi=2.0, idx=np.array([src]), val=np.array([1.0])),
            W.Column(kind="dense", zlo=0.0, zhi=0.5, dense=rng.standard_normal(n)),
            W.Column(kind="box", zlo=0.9, zhi=1.1, box_lo=(0, 0, 0), box_hi=(4, 3, 2), value=2.0)]
    rp, cc, cv = W._c_rows([([src], [1.0]), (np.arange(0, n, 7), rng.standard_normal(len(range(0, n, 7))))])
    mk = lambda prec: W.Problem(system=sysm, columns=cols, C_row_ptr=rp, C_col=cc, C_val=cv,
                                theta=np.array([math.inf, math.inf]), dt=0.02, steps=80, m=20, precision=prec)
    U = np.array([[-1.0, 0.3], [0.5, -1.0]])
    v = np.array([-0.4, 0.2]) + 0.6 * np.linalg.norm(U, axis=1)   # the wedge becomes reachable mid-horizon
    Iz = np.array([[1.0, 1.0, 0.0]])
    iota = np.array([1.5])
    B, zlo, zhi, ref = oracle_lp(mk("fp64"), U, v, Iz, iota)
    assert 0 < ref["viol_step"] < 80
    _, got = gpu_lp(ctx, mk(precision), U, v, Iz, iota)
    compare(got, ref, 1e-9 if precision == "fp64" else 1e-6, B, zlo, zhi, U, v, Iz, iota)
    k = ref["viol_step"]
    scale = np.max(np.abs(ref["margin"]))
    if abs(ref["margin"][k]) > 1e-5 * scale and abs(ref["margin"][k - 1]) > 1e-5 * scale:
        assert got["viol_step"] == k
