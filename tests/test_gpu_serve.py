"""Continuous-batching server (kv_server_*, kv_submit, kv_poll).

Each result must be the same alone and in the mix: queries run on their own
streams with their own device memory and deterministic reductions, so the
bounds are compared bit for bit -- against the same query served alone, and
against kv_run.  FP32 results are also checked against the FP64 oracle
(<= 1e-6 scale-normalised).
"""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from parity import bound_error

pytestmark = pytest.mark.gpu

kv = pytest.importorskip("paper_1804_01583_gb300")


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_01583_gb300 import build as kvbuild
    kvbuild.build()
    return kv.load()


def small_mix(n=16, seed=3):
    return W.serving_mix(n, seed=seed, side2d=(40, 200), side3d=(20, 48), csr_n=(5000, 20000), steps=(50, 300),
                         m=(10, 30))


def wait_all(server, tickets, timeout=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = server.poll(t)
                if r is not None:
                    out[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError("server did not finish")
        time.sleep(0.001)
    return [out[t] for t in tickets]


def test_results_identical_alone_and_in_mix(lib):
    qs = small_mix()
    # alone: one slot, each query waited for before the next is submitted
    ctx1 = kv.Context(8 << 30)
    s1 = kv.Server(ctx1, slots=1)
    alone = []
    for q in qs:
        alone += wait_all(s1, [s1.submit(q)])
    s1.close()
    ctx1.close()
    # in the mix: 8 slots, everything submitted at once
    ctx2 = kv.Context(8 << 30)
    s2 = kv.Server(ctx2, slots=8)
    mixed = wait_all(s2, [s2.submit(q) for q in qs])
    st = s2.stats()
    s2.close()
    ctx2.close()
    assert st["completed"] == len(qs) and st["max_running"] > 1
    # kv_run on the same queries
    ctx3 = kv.Context(8 << 30)
    for q, a, b in zip(qs, alone, mixed):
        assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"]), q.name
        assert a["viol_step"] == b["viol_step"] and np.array_equal(a["m_used"], b["m_used"])
        ref = kv.solve(q, ctx3, expm_mode="propagate")
        assert np.array_equal(ref["hi"], b["hi"]) and np.array_equal(ref["lo"], b["lo"]), q.name
    ctx3.close()


def test_served_error_against_fp64_oracle(lib):
    """The served mix (CSR queries in FP32 storage, heat queries in FP64)
    against the FP64 oracle: within 1e-6 (FP32 storage) and 1e-9 (FP64).
    The heat queries forced to FP32 storage stay under the floor documented
    for the Lanczos recurrence with float vectors (3e-6; 1.0e-6 measured on
    q1 here), which is why the mix serves them in FP64."""
    qs = small_mix(8, seed=11)
    ctx = kv.Context(8 << 30)
    s = kv.Server(ctx, slots=4)
    res = wait_all(s, [s.submit(q) for q in qs])
    s.close()
    n_heat = 0
    for q, r in zip(qs, res):
        q64 = W.Problem(**{**q.__dict__, "precision": "fp64"})
        ref = oracle.run(q64)
        assert bound_error(r, ref) <= (1e-9 if q.precision == "fp64" else 1e-6), q.name
        assert r["latency_ms"] > 0
        if "heat" in q.name:
            n_heat += 1
            r32 = kv.solve(W.Problem(**{**q.__dict__, "precision": "fp32"}), ctx)
            assert bound_error(r32, ref) <= 3e-6, q.name
    ctx.close()
    assert n_heat > 0


def test_admission_waits_for_memory(lib):
    """A pool that holds only a few of the queries at once: later queries wait
    for running ones to release memory, and all complete."""
    qs = [W.heat((64, 64, 64), block=(6, 6, 6), output="centre", dt=0.02, steps=100, m=20, precision="fp32")
          for _ in range(10)]
    ctx = kv.Context(10 << 20)  # ~3 MB per query (three 1 MB vectors + state)
    s = kv.Server(ctx, slots=8)
    res = wait_all(s, [s.submit(q) for q in qs])
    st = s.stats()
    s.close()
    ctx.close()
    assert st["completed"] == 10 and st["memory_waits"] > 0 and st["max_running"] < 8
    for r in res[1:]:
        assert np.array_equal(r["hi"], res[0]["hi"])


def test_query_larger_than_the_pool_fails_and_server_continues(lib):
    ctx = kv.Context(4 << 20)
    s = kv.Server(ctx, slots=2)
    big = W.heat((200, 200, 200), block=(4, 4, 4), output="centre", dt=0.02, steps=10, m=5, precision="fp32")
    ok = W.heat((24, 24), block=(3, 3), output="centre", dt=0.1, steps=10, m=5, precision="fp32")
    tb = s.submit(big)
    to = s.submit(ok)
    t0 = time.time()
    err = None
    while True:
        try:
            r = s.poll(tb)
        except kv.KvError as e:
            err = e
            break
        assert r is None and time.time() - t0 < 60
        time.sleep(0.001)
    assert err.code == kv.KV_ENOMEM
    assert wait_all(s, [to])[0]["hi"].shape == (1, 11)
    s.close()
    ctx.close()


def test_unknown_ticket(lib):
    ctx = kv.Context(1 << 20)
    s = kv.Server(ctx, slots=1)
    q = W.heat((8, 8), block=(2, 2), output="centre", dt=0.1, steps=4, m=4)
    t = s.submit(q)
    wait_all(s, [t])
    res = kv.kv_result()
    out = np.zeros(5)
    res.lo = out.ctypes.data
    res.hi = out.ctypes.data
    rc = lib.kv_poll(s.h, 987654321, res, None)
    assert rc == kv.KV_EINVAL
    s.close()
    ctx.close()


def test_poll_without_outputs_keeps_the_result(lib):
    """A finished query polled without lo/hi is refused (KV_EINVAL) and its
    result stays pollable."""
    ctx = kv.Context(1 << 20)
    s = kv.Server(ctx, slots=1)
    q = W.heat((8, 8), block=(2, 2), output="centre", dt=0.1, steps=4, m=4)
    t = s.submit(q)
    res = kv.kv_result()  # lo and hi left NULL
    t0 = time.time()
    while True:
        rc = lib.kv_poll(s.h, t, res, None)
        if rc != kv.KV_ENOTREADY:
            break
        assert time.time() - t0 < 60
        time.sleep(0.001)
    assert rc == kv.KV_EINVAL
    r = wait_all(s, [t])[0]
    assert r["lo"].shape == (1, 5) and np.all(r["hi"] >= r["lo"])
    s.close()
    ctx.close()


def test_csr_queries_share_one_system_copy(lib):
    """Queries on one CSR system (direct and transpose dynamics, FP32 and FP64
    storage) submitted together: one device copy per storage precision is
    built, the other admissions reuse it, nothing stays resident after they
    finish, and every result equals kv_run's on a system of its own."""
    sysm = W.random_csr(6000, seed=77)
    qs = [W.csr_problem_on(sysm, seed=s, n_gen=g, o=2, c_width=500, dt=0.01, steps=80, m=16, precision=p)
          for s, (g, p) in enumerate([(1, "fp32"), (12, "fp32"), (3, "fp64"), (1, "fp32"), (20, "fp64"),
                                      (5, "fp32")])]
    ctx = kv.Context(2 << 30)
    s = kv.Server(ctx, slots=4)
    res = wait_all(s, [s.submit(q) for q in qs])
    st = s.stats()
    s.close()
    assert st["completed"] == len(qs)
    assert st["systems_built"] == 2 and st["systems_reused"] == len(qs) - 2, st
    assert st["systems_released"] == 0 and st["systems_resident"] == 0, st
    for q, r in zip(qs, res):
        ref = kv.solve(q, ctx, expm_mode="propagate")
        assert np.array_equal(ref["lo"], r["lo"]) and np.array_equal(ref["hi"], r["hi"]), q.name
    ctx.close()


def test_idle_shared_system_released_when_the_pool_is_full(lib):
    """One slot and a pool that holds one CSR system and a query but not two
    systems: after the first query on A, A stays for the third query (also on
    A), and the query on B finds the pool full; A's idle copy is released to
    admit it and rebuilt for the third query.  All results equal kv_run's."""
    A = W.random_csr(60000, seed=5)
    B = W.random_csr(60000, seed=6)
    qa = W.csr_problem_on(A, seed=1, n_gen=1, o=2, c_width=500, dt=0.01, steps=40, m=8, precision="fp32")
    qb = W.csr_problem_on(B, seed=2, n_gen=1, o=2, c_width=500, dt=0.01, steps=40, m=8, precision="fp32")
    qa2 = W.csr_problem_on(A, seed=3, n_gen=1, o=2, c_width=500, dt=0.01, steps=40, m=8, precision="fp32")
    # size the pool from the probe: the larger system, the larger problem, half a system of slack
    probe = kv.Context(1 << 30)
    used0 = probe.pool_stats()[0]
    sys_bytes, prob_bytes = 0, 0
    for q in (qa, qb, qa2):
        h = kv.System(probe, q.system, precision=q.precision)
        sys_bytes = max(sys_bytes, probe.pool_stats()[0] - used0)
        prob_bytes = max(prob_bytes, kv.problem_bytes(h, q, expm_mode="propagate"))
        h.close()
    probe.close()
    pool = sys_bytes + prob_bytes + sys_bytes // 2 + (1 << 20)
    ctx = kv.Context(pool)
    s = kv.Server(ctx, slots=1)
    res = wait_all(s, [s.submit(q) for q in (qa, qb, qa2)])
    st = s.stats()
    s.close()
    assert st["completed"] == 3 and st["systems_released"] >= 1, (st, sys_bytes, prob_bytes)
    assert st["systems_resident"] == 0
    ctx2 = kv.Context(1 << 30)
    for q, r in zip((qa, qb, qa2), res):
        ref = kv.solve(q, ctx2, expm_mode="propagate")
        assert np.array_equal(ref["lo"], r["lo"]) and np.array_equal(ref["hi"], r["hi"])
    ctx2.close()
    ctx.close()


def test_served_grid_with_face_coefficients(lib):
    """A grid system with face coefficients (the paper's heat model: insulated
    faces and one exchange face) is served as that system: the result equals
    kv_run's and differs from the Dirichlet-0 grid of the same sizes."""
    q = W.paper_heat_grid(24, dt=0.02, steps=60, m=24)
    d0 = W.Problem(**{**q.__dict__, "system": W.GridSystem(dims=q.system.dims, coef=q.system.coef,
                                                            h=q.system.h)})
    ctx = kv.Context(1 << 30)
    s = kv.Server(ctx, slots=2)
    r, rd = wait_all(s, [s.submit(q), s.submit(d0)])
    s.close()
    ref = kv.solve(q, ctx, expm_mode="propagate")
    ctx.close()
    assert np.array_equal(ref["lo"], r["lo"]) and np.array_equal(ref["hi"], r["hi"])
    assert not np.array_equal(rd["hi"], r["hi"])
