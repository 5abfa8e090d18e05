"""The allocation-free grid Lanczos entry point (kv_grid_lanczos_noalloc).

It exists for callers that cannot allocate device memory when they need a
result (graph capture in progress, hosts that reserve all device memory up
front).  Its H, P, beta0 and m_used must equal those of the pooled entry point
kv_run on the same problem, within the FP64 parity tolerance, on two
different problems run back to back: the shared scratch array keeps the first
call's contents and the second call must not depend on them.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

kv = pytest.importorskip("paper_1804_01583_gb300")

TOL = 1e-9


def _device_call(p, torch):
    dev = torch.device("cuda:0")
    s = p.system
    col = p.columns[0]
    m, o = p.m, p.o
    crp = torch.tensor(np.asarray(p.C_row_ptr, dtype=np.int64), device=dev)
    ccol = torch.tensor(np.asarray(p.C_col, dtype=np.int64), device=dev)
    cval = torch.tensor(np.asarray(p.C_val, dtype=np.float64), device=dev)
    H = torch.full(((m + 1) * m,), float("nan"), dtype=torch.float64, device=dev)
    P = torch.full((o * m,), float("nan"), dtype=torch.float64, device=dev)
    b0 = torch.zeros(1, dtype=torch.float64, device=dev)
    mu = torch.zeros(1, dtype=torch.int32, device=dev)
    kv.grid_lanczos_noalloc(0, None, len(s.dims), s.dims, s.coef, s.h, col.box_lo, col.box_hi, col.value, o,
                            crp.data_ptr(), ccol.data_ptr(), cval.data_ptr(), m, H.data_ptr(), P.data_ptr(),
                            b0.data_ptr(), mu.data_ptr())
    torch.cuda.synchronize()
    return (H.cpu().numpy().reshape(m + 1, m), P.cpu().numpy().reshape(o, m), float(b0.item()), int(mu.item()))


def _compare(p, ref, got):
    H, P, b0, mu = got
    assert mu == int(ref["m_used"][0])
    Hr = ref["H"][0][: mu + 1, :mu]
    assert np.max(np.abs(H[: mu + 1, :mu] - Hr)) <= TOL * np.max(np.abs(Hr))
    Pr = ref["P"][0][:, :mu]
    sp = np.max(np.abs(Pr))
    if sp == 0.0:
        assert np.all(P[:, :mu] == 0.0)
    else:
        assert np.max(np.abs(P[:, :mu] - Pr)) <= TOL * sp
    assert abs(b0 - ref["beta0"][0]) <= 1e-14 * ref["beta0"][0]


def test_noalloc_matches_pooled_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_01583_gb300 import build as kvbuild
    kvbuild.build()
    # two different problems in a row: a 3D grid with the output in reach,
    # then the 20 x 20 2D heat grid (5 x 5 block, centre output, m = 30)
    p1 = W.heat((40, 30, 20), block=(6, 5, 4), output="centre8", dt=0.02, steps=10, m=25)
    p1.C_col = np.array([W.grid_index((40, 30, 20), (8, 7, 6))], dtype=np.int64)
    p1.C_val = np.array([1.0])
    p1.C_row_ptr = np.array([0, 1], dtype=np.int64)
    p2 = W.heat2d_20(steps=10)
    for p in (p1, p2):
        ref = kv.solve(p, pool_bytes=256 << 20)
        _compare(p, ref, _device_call(p, torch))


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    p = W.heat((100, 100, 100), block=(4, 4, 4), output="centre", dt=0.02, steps=2, m=4)
    buf = torch.zeros(64, dtype=torch.float64, device="cuda:0")
    crp = torch.zeros(2, dtype=torch.int64, device="cuda:0")
    mu = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    with pytest.raises(kv.KvError) as ei:
        kv.grid_lanczos_noalloc(0, None, 3, p.system.dims, p.system.coef, p.system.h, (0, 0, 0), (4, 4, 4), 1.0,
                                1, crp.data_ptr(), crp.data_ptr(), buf.data_ptr(), 4, buf.data_ptr(),
                                buf.data_ptr(), buf.data_ptr(), mu.data_ptr())
    assert ei.value.code == kv.KV_EINVAL
    assert "KV_NOALLOC_MAX_N" in str(ei.value)
