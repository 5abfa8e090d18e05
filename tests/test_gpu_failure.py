"""The failure path of the device waits, on the GPU without a fault: a block
waits on an mbarrier nothing completes, with the single-pass grid kernel's
own bounded-wait routine; the wait expires, the status reaches the host as
KV_ETIMEOUT, and the device stays usable (a problem runs right after and
matches the oracle)."""
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
    c = kv.Context(1 << 30)
    yield c
    c.close()


@pytest.mark.parametrize("polls", [1, 64, 4096])
def test_bounded_wait_expires_and_reports(ctx, polls):
    assert kv.diag_bounded_wait(polls) == kv.KV_ETIMEOUT
    assert "expired" in kv.last_error()
    # the context still works: the FP32 single-pass iteration (the kernel
    # whose waits these are) runs and matches the oracle
    p = W.heat2d_20(theta=0.01, precision="fp32")
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p)
    got = ph.run()
    ph.close()
    sysh.close()
    assert bound_error(got, oracle.run(W.heat2d_20(theta=0.01))) <= 1e-6


def test_bad_poll_counts_rejected(ctx):
    for polls in (0, -5, (1 << 22) + 1):
        assert kv.diag_bounded_wait(polls) == kv.KV_EINVAL
