"""The paper's 3-D heat benchmark (Sec. 5.3, the cell-centred reading of its
insulated cube with heat exchange at x = 1) on the GPU: CSR Lanczos at a
fixed Krylov dimension and under the Lemma-1 error control against the
oracle (H, P and bounds within 1e-9; the same stop dimension and bound), the
library's precision choice routing this operator to FP64, the measured
FP32-storage floor that makes it do so, and the paper's own experiment
(100^3 cells, target 1e-6, T = 20 in 1000 steps) against the exact
separable solution, which the result must meet within its own Lemma-1
bound."""
import numpy as np
import pytest

import oracle
import workloads as W
from parity import bound_error, krylov_error
from test_gpu_errbound import check_control, pick_target
from test_oracle_paper_heat import closed_form

pytestmark = pytest.mark.gpu

kv = pytest.importorskip("paper_1804_01583_gb300")


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_01583_gb300 import build as kvbuild
    kvbuild.build()
    c = kv.Context(16 << 30)
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


@pytest.mark.parametrize("precision", ["fp64", "auto"])
def test_fixed_dimension(ctx, precision):
    """40^3 cells, m = 100, T = 20 in 200 steps: FP64, and the library's
    precision choice (KV_PREC_AUTO), which routes this operator to FP64
    storage (symmetric, mu T = 0 > -1: a slow mode that keeps FP32 rounding
    to the end of the horizon) and so meets 1e-9, below the 1e-6 bar of the
    precision form."""
    p64 = W.paper_heat(40, dt=0.1, steps=200, m=100)
    ref = oracle.run(p64)
    got = run_gpu(ctx, W.paper_heat(40, dt=0.1, steps=200, m=100, precision=precision))
    assert int(got["m_used"][0]) == int(ref["used"][0])
    eh, ep = krylov_error(got, ref, 0)
    assert eh <= 1e-9 and ep <= 1e-9, (eh, ep)
    assert bound_error(got, ref) <= 1e-9


def test_fp32_storage_floor(ctx):
    """FP32 storage forced on the insulated cube: its measured floor, above
    the 1e-6 bar (1.5e-6 here; Lanczos with float vectors and double dot
    products gives 2.5e-6 in numpy), which is why KV_PREC_AUTO routes this
    operator to FP64.  A regression guard on the documented floor, not a
    parity claim."""
    ref = oracle.run(W.paper_heat(40, dt=0.1, steps=200, m=100))
    got = run_gpu(ctx, W.paper_heat(40, dt=0.1, steps=200, m=100, precision="fp32"))
    assert bound_error(got, ref) <= 3e-6


def test_error_control(ctx):
    """20^3 cells, T = 20 in 50 steps: the dimension the control stops at
    (above 64: the global-memory exponential) and the Lemma-1 bound there."""
    p = W.paper_heat(20, dt=0.4, steps=50, m=160)
    p.err_target, (k,) = pick_target(p, near=1e-6)
    ref = oracle.run(p)
    assert ref["used"][0] == k and 64 < k < 160
    got = run_gpu(ctx, p)
    check_control(got, ref, p, 1e-9, 1e-9)


@pytest.mark.parametrize("precision", ["fp64", "auto"])
def test_paper_experiment_against_the_exact_solution(ctx, precision):
    """Sec. 5.3: 100^3 cells, error target 1e-6, T = 20 by 0.02.  The error
    control stops at k = 544, the dimension the paper reports; the centre
    temperature (per unit initial temperature) is within its own Lemma-1
    bound (times ||C|| ||E||) of the exact separable solution at every step
    (measured: 2.3e-7 of the peak in FP64).  KV_PREC_AUTO runs this operator
    in FP64 (FP32 storage would add 2.1e-6 of rounding, measured)."""
    p = W.paper_heat(100, precision=precision, err_target=1e-6)
    got = run_gpu(ctx, p, expm_mode="propagate")
    y = closed_form(100, p.dt, p.steps)
    k = int(got["m_used"][0])
    assert k == 544   # the Krylov dimension the paper reports for this experiment (Sec. 5.3)
    b0 = float(got["beta0"][0])
    allowed = b0 * np.sqrt(8 * 0.125 ** 2) * float(got["err_bound"][0])
    assert float(got["err_bound"][0]) < 1e-6
    err = np.max(np.abs(got["basis"][0][0] - y))
    assert err <= allowed + 1e-9 * np.max(y), (err, allowed)
