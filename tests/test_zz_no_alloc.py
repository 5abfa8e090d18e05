"""The allocation-free grid Lanczos entry point (kv_grid_lanczos_noalloc).

It exists for callers that cannot allocate device memory when they need a
result: hosts that reserve all device memory up front, callers running inside
another runtime's allocator.  Its H, P, beta0 and m_used must equal the CPU
oracle's and those of the pooled entry point kv_run on the same problem,
within the FP64 parity tolerance, on two different problems run back to back:
the shared scratch array keeps the first call's contents and the second call
must not depend on them.  C arrays that point outside the grid are rejected
by the first kernel before anything is read through them.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

kv = pytest.importorskip("paper_1804_01583_gb300")

TOL = 1e-9


def _buffers(p, torch):
    dev = torch.device("cuda:0")
    m, o = p.m, p.o
    return dict(
        crp=torch.tensor(np.asarray(p.C_row_ptr, dtype=np.int64), device=dev),
        ccol=torch.tensor(np.asarray(p.C_col, dtype=np.int64), device=dev),
        cval=torch.tensor(np.asarray(p.C_val, dtype=np.float64), device=dev),
        H=torch.full(((m + 1) * m,), float("nan"), dtype=torch.float64, device=dev),
        P=torch.full((max(o, 1) * m,), float("nan"), dtype=torch.float64, device=dev),
        b0=torch.zeros(1, dtype=torch.float64, device=dev),
        mu=torch.zeros(1, dtype=torch.int32, device=dev),
    )


def _device_call(p, torch, bufs=None):
    s = p.system
    col = p.columns[0]
    m, o = p.m, p.o
    b = bufs if bufs is not None else _buffers(p, torch)
    kv.grid_lanczos_noalloc(0, None, len(s.dims), s.dims, s.coef, s.h, col.box_lo, col.box_hi, col.value, o,
                            b["crp"].data_ptr(), b["ccol"].data_ptr(), b["cval"].data_ptr(), m, b["H"].data_ptr(),
                            b["P"].data_ptr(), b["b0"].data_ptr(), b["mu"].data_ptr())
    torch.cuda.synchronize()
    return (b["H"].cpu().numpy().reshape(m + 1, m), b["P"].cpu().numpy()[: o * m].reshape(o, m),
            float(b["b0"].item()), int(b["mu"].item()))


def _compare(ref, got):
    H, P, b0, mu = got
    # the pooled entry point reports m_used, the oracle `used` (per column)
    assert mu == int((ref["m_used"] if "m_used" in ref else ref["used"])[0])
    Hr = np.asarray(ref["H"][0])[: mu + 1, :mu]
    assert np.max(np.abs(H[: mu + 1, :mu] - Hr)) <= TOL * np.max(np.abs(Hr))
    Pr = np.asarray(ref["P"][0])[:, :mu]
    sp = np.max(np.abs(Pr))
    if sp == 0.0:
        assert np.all(P[:, :mu] == 0.0)
    else:
        assert np.max(np.abs(P[:, :mu] - Pr)) <= TOL * sp
    assert abs(b0 - ref["beta0"][0]) <= 1e-14 * ref["beta0"][0]


def _problems():
    # a 3D grid with the output in reach, then the 20 x 20 2D heat grid
    # (5 x 5 block, centre output, m = 30)
    p1 = W.heat((40, 30, 20), block=(6, 5, 4), output="centre8", dt=0.02, steps=10, m=25)
    p1.C_col = np.array([W.grid_index((40, 30, 20), (8, 7, 6))], dtype=np.int64)
    p1.C_val = np.array([1.0])
    p1.C_row_ptr = np.array([0, 1], dtype=np.int64)
    p2 = W.heat2d_20(steps=10)
    return p1, p2


def _torch_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1804_01583_gb300 import build as kvbuild
    kvbuild.build()
    return torch


def test_noalloc_matches_oracle_and_pooled_entry_point_on_two_calls():
    import oracle
    torch = _torch_gpu()
    for p in _problems():
        got = _device_call(p, torch)
        _compare(oracle.run(p), got)
        _compare(kv.solve(p, pool_bytes=256 << 20), got)


def test_noalloc_allocates_nothing_after_the_first_call():
    torch = _torch_gpu()
    p = _problems()[1]
    bufs = _buffers(p, torch)
    _device_call(p, torch, bufs)  # first call on the device: symbol look-up, module load
    dev_before = torch.cuda.current_device()
    free0, _ = torch.cuda.mem_get_info()
    got = _device_call(p, torch, bufs)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.current_device() == dev_before
    assert got[3] == p.m


def test_noalloc_rejects_C_outside_the_grid_before_reading_it():
    torch = _torch_gpu()
    p = _problems()[1]
    n = int(np.prod(p.system.dims))
    bad = _buffers(p, torch)
    bad["ccol"].fill_(n)  # one past the last grid point
    H, P, b0, mu = _device_call(p, torch, bad)
    assert mu == -1
    assert np.all(H == 0.0) and np.all(P == 0.0)
    # the scratch array is not left in a state the next call depends on
    _compare(kv.solve(p, pool_bytes=256 << 20), _device_call(p, torch))


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = _torch_gpu()
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
    with pytest.raises(kv.KvError) as ei:  # C arrays missing while o > 0
        kv.grid_lanczos_noalloc(0, None, 2, (20, 20), 0.01, (1 / 21, 1 / 21), (0, 0), (5, 5), 1.0, 1,
                                crp.data_ptr(), None, None, 4, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                mu.data_ptr())
    assert ei.value.code == kv.KV_EINVAL
