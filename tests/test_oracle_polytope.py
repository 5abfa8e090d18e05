"""Pins of the oracle's per-step LP for polyhedral sets (Sec. 2.1 with the
output and initial spaces of Sec. 3.1-3.2): the paper's worked LP on the
harmonic oscillator, the closed form of one half-space (which equals the
box-bound path), brute-force vertex enumeration on small cases, and the
empty initial set."""
import itertools
import json
import math
import os

import numpy as np

import oracle
import workloads as W
from oracle import polytope as LP


def oscillator_full_state():
    """The oscillator with C = I on (x, y, t): the basis is the 3 x 2 block of
    e^{A t_k} E, so B_k z is the state reached from z = (y0, 1)."""
    p = W.oscillator()
    p.C_row_ptr, p.C_col, p.C_val = W._c_rows([([0], [1.0]), ([1], [1.0]), ([2], [1.0])])
    p.theta = np.full(3, np.inf)
    return p


def test_oscillator_lp_worked_example(golden_dir):
    """Sec. 2.2: with the unsafe set x = 4 the LP is infeasible at steps 0,
    pi/4 and pi/2 and feasible at 3 pi/4, from (x0, y0) = (-5, 0.66) to the
    state (4, 3.07, 2.36) (the constant variable stays 1)."""
    g = json.load(open(os.path.join(golden_dir, "oscillator.json")))
    tol = g["printed_digits_tol"]
    p = oscillator_full_state()
    r = oracle.run(p)
    U = np.array([[1.0, 0, 0], [-1.0, 0, 0]])    # x <= 4 and x >= 4
    v = np.array([4.0, -4.0])
    basis = np.stack([r["basis"][j] for j in range(p.i)])    # [j][r][k]
    res = LP.check(basis, [0.0, 1.0], [1.0, 1.0], U, v, tol=1e-9)
    assert res["viol_step"] == g["violation_step"]
    for k in g["no_violation_steps"]:
        assert res["margin"][k] > 1.0
    z = res["z_star"]
    assert abs(z[0] - g["lp_initial_point"][1]) < tol and z[1] == 1.0
    x0 = np.array([-5.0 * z[1], z[0], 0.0])      # E z on (x, y, t)
    assert np.max(np.abs(x0 - np.array(g["lp_initial_point"][:3]))) < tol
    assert np.max(np.abs(res["y_star"] - np.array(g["lp_final_point"][:3]))) < tol
    # closed form of the margin: the distance from 4 to the x-interval
    # {-5 cos t + y0 sin t : y0 in [0, 1]} at t = k pi / 4
    for k in range(5):
        t = k * math.pi / 4
        a, b = sorted([-5 * math.cos(t), -5 * math.cos(t) + math.sin(t)])
        want = max(a - 4.0, 4.0 - b, 0.0)
        assert abs(res["margin"][k] - want) < 1e-12, (k, res["margin"][k], want)


def random_basis(rng, i, o, S):
    return rng.standard_normal((i, o, S)) * np.exp(rng.uniform(-2, 1, size=(1, 1, S)))


def test_one_halfspace_is_the_interval_bound():
    """One unsafe row y_r >= theta (U = -e_r): t*_k = theta - hi_r(k), and
    y_r <= theta: t*_k = lo_r(k) - theta, with hi and lo the box bounds of
    the closed-form path (pinned to the paper elsewhere)."""
    rng = np.random.default_rng(0)
    i, o, S = 5, 3, 9
    B = random_basis(rng, i, o, S)
    zlo = rng.uniform(-1, 0, i)
    zhi = zlo + rng.uniform(0, 2, i)
    theta = rng.standard_normal(o)
    b = oracle.bounds(B, zlo, zhi, theta)
    for r in range(o):
        e = np.zeros(o)
        e[r] = 1.0
        up = LP.check(B, zlo, zhi, -e[None, :], [-theta[r]])
        assert np.allclose(up["margin"], theta[r] - b["hi"][r], rtol=0, atol=1e-12)
        dn = LP.check(B, zlo, zhi, 3.0 * e[None, :], [3.0 * theta[r]])   # scaled row: same half-space
        assert np.allclose(dn["margin"], b["lo"][r] - theta[r], rtol=0, atol=1e-12)


def brute_force(B, zlo, zhi, U, v, Iz, iota):
    """min t over the vertices of {(z, t): Un B z - t <= vn, I_z z <= iota,
    lo <= z <= hi}: every choice of i+1 active constraints."""
    o, i = B.shape
    Un, vn = LP.normalise(U, v)
    A = [np.append(Un[u] @ B, -1.0) for u in range(len(vn))]
    b = list(vn)
    for q in range(len(iota)):
        A.append(np.append(Iz[q], 0.0))
        b.append(iota[q])
    for j in range(i):
        e = np.zeros(i + 1)
        e[j] = 1.0
        A += [e, -e]
        b += [zhi[j], -zlo[j]]
    A, b = np.array(A), np.array(b)
    best = np.inf
    for act in itertools.combinations(range(len(b)), i + 1):
        M = A[list(act)]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, b[list(act)])
        if np.all(A @ x <= b + 1e-9):
            best = min(best, x[-1])
    return best


def test_brute_force_vertices():
    rng = np.random.default_rng(1)
    for trial in range(12):
        i, o, S = 2 + trial % 2, 2, 4
        B = random_basis(rng, i, o, S)
        zlo = rng.uniform(-1, 0, i)
        zhi = zlo + rng.uniform(0.2, 2, i)
        U = rng.standard_normal((3, o))
        v = rng.standard_normal(3)
        Iz = rng.standard_normal((1, i))
        iota = np.array([Iz[0] @ (zlo + zhi) / 2 + 0.1])   # keeps the box centre inside
        res = LP.check(B, zlo, zhi, U, v, Iz, iota)
        for k in range(S):
            want = brute_force(B[:, :, k].T, zlo, zhi, U, v, Iz, iota)
            assert abs(res["margin"][k] - want) < 1e-9 * max(1.0, abs(want)), (trial, k)
            # the minimiser is in the initial set and meets the unsafe rows relaxed by t*
            assert LP.feasible(B[:, :, k].T, zlo, zhi, U, v + res["margin"][k] * np.linalg.norm(U, axis=1),
                               Iz, iota, res["z"][k], 1e-9)


def test_brute_force_small_basis():
    """A basis of size ~1e-9 (early steps of a heat problem): the unsafe
    rows' z coefficients are tiny next to the t coefficient, and the margin
    still matches the vertices to 1e-12."""
    rng = np.random.default_rng(3)
    for trial in range(40):
        i, o = 1 + trial % 4, 1 + trial % 3
        B = rng.standard_normal((o, i)) * 1e-9
        zlo = rng.uniform(-1, 0, i)
        zhi = zlo + rng.uniform(0.2, 2, i)
        U = rng.standard_normal((1 + trial % 3, o))
        v = rng.standard_normal(len(U))
        want = brute_force(B, zlo, zhi, U, v, np.zeros((0, i)), np.zeros(0))
        st, t, z = LP.step_lp(B, zlo, zhi, U, v)
        assert st == LP.OPTIMAL and abs(t - want) < 1e-12 * max(1.0, abs(want)), (trial, t, want)


def test_empty_initial_set():
    rng = np.random.default_rng(2)
    B = random_basis(rng, 3, 2, 5)
    zlo, zhi = np.zeros(3), np.ones(3)
    res = LP.check(B, zlo, zhi, np.array([[1.0, 1.0]]), [0.0], Iz=np.array([[1.0, 1.0, 1.0]]), iota=[-0.5])
    assert np.all(res["status"] == LP.EMPTY) and res["viol_step"] == -1
