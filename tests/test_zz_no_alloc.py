"""The allocation-free linked-cell sort, for callers that cannot allocate
device memory while they run (a program that gave the whole device to its own
pool allocator, or a time-stepping loop that must not allocate once it is
running).  It must give exactly what the allocating sort gives -- integer
work, so bit for bit -- on consecutive calls that reuse its fixed scratch
array, through the C ABI with caller-owned device buffers."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_00336_gb300 import build, dps
    build.build()
    L = dps.lib()
    vp = ctypes.c_void_p
    L.dps_op_cell_sort_noalloc.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                           ctypes.c_int64, vp, vp, vp, vp, vp]
    return torch, dps, L


def _noalloc(torch, L, n, per, x, ids):
    ncell = n[0] * n[1] * n[2]
    cs = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
    order = torch.full((max(len(ids), 1),), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    rc = L.dps_op_cell_sort_noalloc((ctypes.c_int * 3)(*n), (ctypes.c_int * 3)(*per), 1, len(ids),
                                    ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(ids.data_ptr()),
                                    ctypes.c_void_p(cs.data_ptr()), ctypes.c_void_p(order.data_ptr()),
                                    ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize()
    return rc, cs, order[:len(ids)]


def test_noalloc_sort_equals_allocating_sort_on_consecutive_calls():
    torch, dps, L = _setup()
    from paper_1711_00336_gb300 import workloads
    cases = [((40, 33, 29), (1, 1, 0), 3000, 6), ((17, 11, 9), (1, 0, 1), 500, 5)]
    for n, per, count, seed in cases:  # the second call reuses the array the first one filled
        pr = workloads.random_particles(n, per, count, seed)
        rng = np.random.default_rng(seed)
        x = torch.tensor(pr["x"], dtype=torch.float64, device="cuda")
        ids = torch.tensor(rng.permutation(count).astype(np.int32), device="cuda")
        cs_ref, order_ref = dps.op_cell_sort(n, per, x, ids)
        torch.cuda.synchronize()
        rc, cs, order = _noalloc(torch, L, n, per, x, ids)
        assert rc == 0
        assert torch.equal(cs, cs_ref)
        assert torch.equal(order, order_ref)


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    torch, dps, L = _setup()
    n = (128, 64, 64)  # 524,288 cells > DPS_NOALLOC_MAX_CELLS
    x = torch.full((1, 3), 1.5, dtype=torch.float64, device="cuda")
    ids = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc, _, _ = _noalloc(torch, L, n, (1, 1, 1), x, ids)
    assert rc == -1  # DPS_ERR_ARG


def _pool_used_high(torch):
    """high-water mark of the device's default stream-ordered memory pool
    (reset to zero by the call), through the CUDA runtime the library uses"""
    rt = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    used_high = 0x8  # cudaMemPoolAttrUsedMemHigh
    v = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, used_high, ctypes.byref(v)) == 0
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0
    return v.value


def test_noalloc_sort_takes_nothing_from_the_stream_ordered_pool_and_handles_no_particles():
    """The allocating sort draws its scratch from the stream-ordered pool (the
    pool's high-water mark rises); the allocation-free one leaves it at zero.
    With no particles it returns all-zero offsets."""
    torch, dps, L = _setup()
    from paper_1711_00336_gb300 import workloads
    n, per = (20, 16, 12), (1, 1, 1)
    pr = workloads.random_particles(n, per, 800, 3)
    x = torch.tensor(pr["x"], dtype=torch.float64, device="cuda")
    ids = torch.arange(800, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    _pool_used_high(torch)  # reset
    dps.op_cell_sort(n, per, x, ids)
    torch.cuda.synchronize()
    assert _pool_used_high(torch) > 0
    rc, cs, order = _noalloc(torch, L, n, per, x, ids)
    assert rc == 0
    assert _pool_used_high(torch) == 0
    rc, cs0, _ = _noalloc(torch, L, n, per, x[:0], ids[:0])
    assert rc == 0 and int(cs0.abs().sum()) == 0
