"""Seeded workload generators: shapes, symmetry, Laplacian structure."""
import numpy as np
import pytest

from workloads import graphs as G


def _check_laplacian(lap):
    a = lap.scipy(with_shift=False)
    assert (a - a.T).nnz == 0
    assert np.allclose(np.asarray(a.sum(axis=1)).ravel(), 0.0)
    assert np.all(np.diff(lap.row_ptr) >= 0) and lap.row_ptr[-1] == lap.nnz
    assert lap.col_idx.min() >= 0 and lap.col_idx.max() < lap.n
    for r in range(0, lap.n, max(1, lap.n // 50)):
        seg = lap.col_idx[lap.row_ptr[r]:lap.row_ptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
    assert np.all(np.abs(lap.values - np.round(lap.values)) == 0)


def test_grid_sizes():
    g2 = G.grid2d(40, 50)
    assert (g2.n, g2.nnz) == (2000, 9820)
    _check_laplacian(g2)
    g3 = G.grid3d(10, 11, 12, 0.01)
    assert g3.nnz == 10 * 11 * 12 + 2 * (9 * 11 * 12 + 10 * 10 * 12 + 10 * 11 * 11)
    _check_laplacian(g3)


def test_knn_and_rgg():
    k = G.knn3d(3000, 10, seed=1)
    _check_laplacian(k)
    deg = np.diff(k.row_ptr) - 1
    assert deg.min() >= 10 and 10 < deg.mean() < 16
    assert k.checksum() == G.knn3d(3000, 10, seed=1).checksum()
    assert k.checksum() != G.knn3d(3000, 10, seed=2).checksum()
    r = G.rgg2d(2000, seed=0)
    _check_laplacian(r)


def test_sbm():
    s = G.sbm([300, 500, 200], 20 / 300, 1 / 1000, seed=4)
    _check_laplacian(s)
    assert s.n == 1000
    a = s.scipy(with_shift=False)
    within = a[:300, :300].nnz - 300
    across = a[:300, 300:].nnz
    assert within > 5 * across
