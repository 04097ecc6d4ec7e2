"""Allocation-free Gram entry point, checked against rafeast_gram.

Some callers cannot let the library allocate device memory during a call
(their own allocator owns the device memory, or they must not stall on
cudaMalloc/cudaFree). rafeast_gram_noalloc serves them from a fixed device
array compiled into the library. This file is collected last so that a run
stopping at the first failure has already run every other test; it passes
on its own in a fresh process as well as after the others.
"""
import numpy as np
import pytest

from gpu_util import colmajor_dev
from workloads import graphs as G

pytestmark = pytest.mark.gpu


def _device_memory(torch):
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    return free, torch.cuda.memory_allocated()


def _gram_ref(lib, torch, h, m, X, Y):
    ref = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    lib.rafeast_gram(h, m, X, Y, ref)
    return ref.cpu().numpy()


def test_gram_noalloc_matches_gram_on_consecutive_calls(lib):
    """Calls in a row with every kernel variant (m = 64, 23, 40, 8: 4, 2, 3
    and 1 column blocks per thread), and with n shrinking from 2867 rows
    (64 partial sums) to 100 and 5 rows (7 and 1), so partial sums left by
    an earlier, larger call would be summed if they leaked into a later one.
    After the set-up call, no call changes the device's free memory or
    torch's allocation."""
    import torch
    lap = G.grid2d(61, 47)  # n = 2867: many partial blocks and a ragged tail
    n = lap.n
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, 0.0)
    try:
        rng = np.random.default_rng(2024)
        cases = [(n, 64), (n, 23), (n, 40), (n, 8), (100, 40), (5, 64), (100, 8)]
        inputs = []
        for rows, m in cases:
            x = rng.standard_normal((rows, m))
            y = rng.standard_normal((rows, m))
            got = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")
            inputs.append((rows, m, x, y, colmajor_dev(x), colmajor_dev(y), got))
        # references from rafeast_gram (it needs the handle's n rows); the
        # device buffers it wrote are released before the measured calls
        refs = [_gram_ref(lib, torch, h, m, X, Y) if rows == n else None
                for rows, m, x, y, X, Y, _ in inputs]
        # the set-up call (loads the array and the kernels on this device)
        one = torch.ones((1, 1), dtype=torch.float64, device="cuda")
        out = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
        lib.rafeast_gram_noalloc(one, one, 1, 1, out)
        before = _device_memory(torch)
        for (rows, m, x, y, X, Y, got), ref in zip(inputs, refs):
            lib.rafeast_gram_noalloc(X, Y, rows, m, got)
            g = got.cpu().numpy()
            scale = np.abs(x.T @ y).max()
            assert np.abs(g.T - x.T @ y).max() <= 1e-12 * scale, (rows, m)
            if ref is not None:
                assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max(), (rows, m)
        assert _device_memory(torch) == before
        assert float(out.cpu()[0, 0]) == 1.0
    finally:
        lib.rafeast_destroy(h)


def test_gram_noalloc_rejects_too_many_columns(lib):
    import torch
    n, m = 100, 65
    X = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    Gd = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.RafeastError) as err:
        lib.rafeast_gram_noalloc(X, X, n, m, Gd)
    assert err.value.code == lib.RAFEAST_ERR_INVALID_ARG
    assert "64" in lib.load().rafeast_last_error().decode()
