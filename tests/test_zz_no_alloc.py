"""The allocation-free variant of the stable cell sort.

Some callers cannot allocate device memory while they run (a pool or arena
allocator that owns the whole device, a runtime that forbids cudaMalloc after
start-up).  orbc_cell_sort_noalloc serves them with a fixed scratch array in
the library; this checks, through the C ABI, that two calls in a row give the
same permutation and cell offsets as orbc_cell_sort, and that requests beyond
the array's limits are refused.  The file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call(fn, cell, K, torch):
    n = cell.numel()
    perm = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    start = torch.full((K + 1,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(C.c_void_p(cell.data_ptr()), n, K, C.c_void_p(perm.data_ptr()), C.c_void_p(start.data_ptr()),
            C.c_void_p(stream))
    return rc, perm[:n].cpu().numpy(), start.cpu().numpy()


def test_noalloc_matches_allocating_sort_twice():
    torch = pytest.importorskip("torch")
    from paper_1701_02059_gb300 import _native
    L = _native.load()
    rng = np.random.default_rng(11)
    cases = [(300_000, 4096), (70_000, 12)]      # second call: fewer items, big cells, stale scratch
    for n, K in cases:
        cell = rng.integers(0, K, size=n).astype(np.int32)
        if K == 12:
            cell[:5000] = 2                          # a cell beyond the shared-memory sort
        d = torch.from_numpy(cell).cuda()
        rc_a, perm_a, start_a = _call(L.orbc_cell_sort, d, K, torch)
        rc_b, perm_b, start_b = _call(L.orbc_cell_sort_noalloc, d, K, torch)
        assert rc_a == 0 and rc_b == 0
        assert np.array_equal(perm_a, perm_b)
        assert np.array_equal(start_a, start_b)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1701_02059_gb300 import _native
    L = _native.load()
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc, _, _ = _call(L.orbc_cell_sort_noalloc, d, 70_000, torch)
    assert rc == _native.ORBC_E_NOMEM
    big = torch.zeros((1 << 20) + 1, dtype=torch.int32, device="cuda")
    rc, _, _ = _call(L.orbc_cell_sort_noalloc, big, 8, torch)
    assert rc == _native.ORBC_E_NOMEM
