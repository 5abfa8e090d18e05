"""Device-side checks that turn bad values into reported errors.

Always on: a Krylov scalar that is not finite (the norm of a column, alpha or
beta) ends the column and kv_fetch reports KV_EINVAL, where a NaN or an
overflow would otherwise pass as a breakdown with silently wrong bounds; an
output-matrix column index outside the state vector is skipped, not read.
The debug build (build.py, debug=True: -DKV_DEBUG) adds the same check on
the matrix and scattered-column indices and a test hook that plants an
out-of-range C index on the device (the host validation refuses one at
kv_problem), so the skip is exercised without any invalid memory access.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

kv = pytest.importorskip("paper_1804_01583_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_01583_gb300 import build as kvbuild
    kvbuild.build()
    c = kv.Context(1 << 30)
    yield c
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_overflowing_operator_is_reported(ctx, precision):
    """coef / h^2 overflows to inf on an otherwise valid grid: the first
    Krylov scalars are not finite, and the problem reports it."""
    sysm = W.GridSystem(dims=(8, 8), coef=1e306, h=(1e-3, 1e-3))
    col = W.Column(kind="box", zlo=0.9, zhi=1.1, box_lo=(0, 0), box_hi=(3, 3), value=1.0)
    rp, cc, cv = W._c_rows([([W.grid_index((8, 8), (4, 4))], [1.0])])
    p = W.Problem(system=sysm, columns=[col], C_row_ptr=rp, C_col=cc, C_val=cv, theta=np.array([np.inf]),
                  dt=0.1, steps=5, m=6, precision=precision)
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p)
    try:
        with pytest.raises(kv.KvError) as ei:
            ph.run()
        assert ei.value.code == kv.KV_EINVAL and "not finite" in str(ei.value)
    finally:
        ph.close()
        sysh.close()
    # the context stays usable
    q = W.heat2d_20(steps=10)
    got = kv.solve(q, ctx)
    assert got["m_used"][0] == q.m


def test_overflowing_csr_lanczos_is_reported(ctx):
    """Symmetric CSR, FP64, every entry 1e308: A v overflows in the CSR
    Lanczos pair, and the non-finite alpha and beta are reported instead of
    passing as a breakdown.  The context stays usable."""
    n = 4
    rp = np.arange(0, n * n + 1, n, dtype=np.int64)
    cols = np.tile(np.arange(n, dtype=np.int32), n)
    sysm = W.CsrSystem(n=n, row_ptr=rp, col=cols, val=np.full(n * n, 1e308), symmetric=True)
    col = W.Column(kind="sparse", zlo=0.9, zhi=1.1, idx=np.arange(n), val=np.ones(n))
    crp, cc, cv = W._c_rows([([0], [1.0])])
    p = W.Problem(system=sysm, columns=[col], C_row_ptr=crp, C_col=cc, C_val=cv, theta=np.array([np.inf]),
                  dt=0.1, steps=5, m=3, precision="fp64")
    sysh = kv.System(ctx, p.system, "fp64")
    ph = kv.ProblemHandle(ctx, sysh, p)
    try:
        with pytest.raises(kv.KvError) as ei:
            ph.run()
        assert ei.value.code == kv.KV_EINVAL and "not finite" in str(ei.value)
    finally:
        ph.close()
        sysh.close()
    base = W.paper_heat(6, dt=0.1, steps=5, m=6)
    from parity import bound_error
    assert bound_error(kv.solve(base, ctx), oracle.run(base)) <= 1e-9


def test_exponential_scaling_beyond_its_range_is_reported(ctx):
    """The global-memory exponential scales dt H by up to 2^32 (32 squaring
    launches, fewer when a bound of ||A|| limits them): a step so long that
    ||dt H||_1 needs more is reported, not truncated.  A step inside the
    range gives the oracle's bounds."""
    p = W.heat2d_20(steps=4, dt=1e9)
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p, expm_mode="propagate")
    try:
        with pytest.raises(kv.KvError) as ei:
            ph.run()
        assert ei.value.code == kv.KV_EINVAL and "squarings" in str(ei.value)
    finally:
        ph.close()
        sysh.close()
    from parity import bound_error
    q = W.heat2d_20(steps=40, dt=5.0)
    assert bound_error(kv.solve(q, ctx, expm_mode="propagate"), oracle.run(q)) <= 1e-9


_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle, workloads as W
import paper_1804_01583_gb300 as kv
from parity import bound_error
p = W.heat2d_20(theta=0.01, steps=60)
n = int(np.prod(p.system.dims))
ctx = kv.Context(1 << 28)
sysh = kv.System(ctx, p.system)
ph = kv.ProblemHandle(ctx, sysh, p)
out = {}
kv.debug_set_c_col(ph, 0, n + 5)            # one C entry past the grid
try:
    ph.run()
    out["bad"] = "no error"
except kv.KvError as e:
    out["bad"] = [e.code, str(e)]
kv.debug_set_c_col(ph, 0, int(p.C_col[0]))  # restored
got = ph.run()
out["restored_err"] = bound_error(got, oracle.run(p))
out["restored_viol"] = [int(got["viol_step"]), int(oracle.run(p)["viol_step"])]
print("RESULT " + json.dumps(out))
"""


def test_debug_build_skips_an_out_of_range_C_index(ctx):
    from paper_1804_01583_gb300 import build as kvbuild
    lib = kvbuild.build(debug=True)
    env = dict(os.environ, KV_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT + os.sep + "tests"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    line = next(s for s in r.stdout.splitlines() if s.startswith("RESULT "))
    out = json.loads(line[len("RESULT "):])
    code, msg = out["bad"]
    assert code == kv.KV_EINVAL and "bounds check" in msg, out
    assert out["restored_err"] <= 1e-9
    assert out["restored_viol"][0] == out["restored_viol"][1]
