"""Small queries packed under one captured CUDA graph (kv_graph_*): the
results of every packed problem equal kv_run's bit for bit, on repeated
launches; the columns of one CSR query share each pass's launch (grid.y =
column) and match the oracle (see test_gpu_csr.py)."""
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
    c = kv.Context(4 << 30)
    yield c
    c.close()


def mixed_small():
    qs = [W.heat2d_20(theta=0.01), W.heat2d_20(precision="fp32", theta=0.01), W.oscillator(),
          W.heat((24, 20, 12), block=(4, 3, 2), output="centre8", dt=0.02, steps=60, m=20),
          W.random_csr_problem(3000, seed=5, n_gen=5, o=2, c_width=600, dt=0.01, steps=200, m=25),
          W.random_csr_problem(2000, seed=6, n_gen=3, o=2, c_width=400, dt=0.01, steps=100, m=15,
                               precision="fp32")]
    qs += W.serving_mix(10, seed=9, side2d=(40, 120), side3d=(20, 32), csr_n=(3000, 8000), steps=(50, 200),
                        m=(10, 25))
    return qs


@pytest.mark.parametrize("expm_mode", ["per_step", "propagate"])
def test_graph_results_equal_kv_run(ctx, expm_mode):
    qs = mixed_small()
    refs = [kv.solve(q, ctx, expm_mode=expm_mode) for q in qs]
    systems = [kv.System(ctx, q.system, q.precision) for q in qs]
    handles = [kv.ProblemHandle(ctx, s, q, expm_mode=expm_mode) for s, q in zip(systems, qs)]
    g = kv.Graph(ctx, handles)
    for _ in range(2):
        g.launch()
        for q, h, r in zip(qs, handles, refs):
            got = h.fetch()
            assert np.array_equal(got["hi"], r["hi"]) and np.array_equal(got["lo"], r["lo"]), q.name
            assert np.array_equal(got["H"], r["H"]) and got["viol_step"] == r["viol_step"], q.name
    g.close()
    for h in handles:
        h.close()
    for s in systems:
        s.close()


def test_graph_fp64_results_match_oracle(ctx):
    qs = [W.heat2d_20(theta=0.01), W.oscillator()]
    systems = [kv.System(ctx, q.system, q.precision) for q in qs]
    handles = [kv.ProblemHandle(ctx, s, q) for s, q in zip(systems, qs)]
    g = kv.Graph(ctx, handles)
    g.launch()
    for q, h in zip(qs, handles):
        got = h.fetch()
        ref = oracle.run(q)
        assert bound_error(got, ref) <= 1e-9 and got["viol_step"] == ref["viol_step"]
    g.close()
    for h in handles:
        h.close()
    for s in systems:
        s.close()


def test_polytope_check_follows_graph_launches(ctx):
    """A problem captured in a graph has not run until the graph is launched:
    the per-step LP refuses it before, and after the launch gives the same
    margins as after kv_run."""
    q = W.oscillator()
    q.C_row_ptr, q.C_col, q.C_val = W._c_rows([([0], [1.0]), ([1], [1.0]), ([2], [1.0])])
    q.theta = np.full(3, np.inf)
    U = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    v = np.array([4.0, -4.0])
    s = kv.System(ctx, q.system, q.precision)
    h = kv.ProblemHandle(ctx, s, q)
    g = kv.Graph(ctx, [h])
    with pytest.raises(kv.KvError) as ei:
        h.check_polytope(U, v, tol=1e-9)
    assert ei.value.code == kv.KV_EINVAL
    g.launch()
    via_graph = h.check_polytope(U, v, tol=1e-9)
    h.run()
    direct = h.check_polytope(U, v, tol=1e-9)
    assert via_graph["viol_step"] == direct["viol_step"] == 3
    assert np.array_equal(via_graph["margin"], direct["margin"])
    g.close()
    h.close()
    s.close()
