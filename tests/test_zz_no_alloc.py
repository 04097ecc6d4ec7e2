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


def test_gram_noalloc_matches_gram_on_consecutive_calls(lib):
    import torch
    lap = G.grid2d(61, 47)  # n = 2867: many partial blocks and a ragged tail
    n = lap.n
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, 0.0)
    try:
        rng = np.random.default_rng(2024)
        # two calls in a row; the second one is smaller, so stale partials of
        # the first call would show up if they were summed
        for m in (64, 23):
            x = rng.standard_normal((n, m))
            y = rng.standard_normal((n, m))
            X, Y = colmajor_dev(x), colmajor_dev(y)
            ref = torch.zeros((m, m), dtype=torch.float64, device="cuda")
            lib.rafeast_gram(h, m, X, Y, ref)
            got = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")
            lib.rafeast_gram_noalloc(X, Y, n, m, got)
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()
            assert np.abs(g.T - x.T @ y).max() <= 1e-12 * np.abs(r).max()
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
