"""The replicated-block shape of Sec. 5.2 (n = 28 h, i = 8 h interval
variables, o = 1 output: the mean of one variable over the copies) with a
seeded stand-in block: the transpose dynamics need one Krylov run instead of
8 h.  GPU against the oracle, forward and transposed; with thousands of
columns the bounds go through the column-chunked reduction."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity import bound_error, check_violation

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


@pytest.mark.parametrize("simulate", ["transpose", "forward"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_replicated_small(ctx, simulate, precision):
    p = W.replicated_blocks(20, simulate=simulate, precision=precision)
    ref = oracle.run(W.replicated_blocks(20, simulate=simulate))
    got = run_gpu(ctx, p, expm_mode="propagate")
    assert got["transposed"] == (simulate == "transpose")
    assert len(got["m_used"]) == (1 if simulate == "transpose" else p.i)
    assert bound_error(got, ref) <= (1e-9 if precision == "fp64" else 1e-6)


def test_replicated_many_columns_chunked_bounds(ctx):
    """h = 3000: i = 24000 columns, one transposed run; a threshold between
    the initial output and its peak makes a violation and a counter-example
    over all 24000 columns."""
    p = W.replicated_blocks(3000)
    ref = oracle.run(p)
    hi = ref["hi"][0]
    p.theta = np.array([0.5 * (hi[0] + np.max(hi))]) if np.max(hi) > hi[0] else np.array([0.9 * hi[0]])
    ref = oracle.run(p)
    got = run_gpu(ctx, p, expm_mode="propagate")
    assert len(got["m_used"]) == 1 and int(got["m_used"][0]) == int(ref["used"][0])
    assert bound_error(got, ref) <= 1e-9
    check_violation(got, ref, p, 1e-9)
