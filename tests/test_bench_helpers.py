"""Host logic of bench.py that needs no GPU: the whole-job rate over ranks is
covered in test_multi_rank.py; here the detection of unit-weight Laplacians,
which decides the values-free byte and FP64-operation counts of the dot
kernel's roofline."""
import numpy as np

import bench
from workloads import graphs as G


def test_unit_laplacians_are_detected():
    for lap in (G.knn3d(300, 6, seed=2, shift=1e-3), G.grid2d(7, 9, 0.0), G.rgg2d(200, seed=1)):
        vf, nnz_off = bench._unit_laplacian(lap)
        assert vf
        rows = np.repeat(np.arange(lap.n), np.diff(lap.row_ptr))
        assert nnz_off == int(np.sum(rows != lap.col_idx))


def test_isolated_vertex_is_still_a_unit_laplacian():
    base = G.knn3d(120, 5, seed=3, shift=0.0).scipy().tocoo()
    keep = (base.row < base.col) & (base.row != 0) & (base.col != 0)
    lap = G._from_edges(120, base.row[keep], base.col[keep], 0.0, "cut")
    assert lap.row_ptr[1] == lap.row_ptr[0]
    assert bench._unit_laplacian(lap)[0]


def test_other_weights_are_not():
    lap = G.grid2d(6, 5, 0.0)
    w = lap.values.copy()
    rows = np.repeat(np.arange(lap.n), np.diff(lap.row_ptr))
    off = np.flatnonzero(rows != lap.col_idx)
    w[off[0]] = -2.0  # one weight other than -1
    bad = G.Laplacian(lap.n, lap.row_ptr, lap.col_idx, w, lap.shift, "w")
    assert not bench._unit_laplacian(bad)[0]
    d = lap.values.copy()
    d[np.flatnonzero(rows == lap.col_idx)[0]] += 0.5  # a diagonal that is not the degree
    bad = G.Laplacian(lap.n, lap.row_ptr, lap.col_idx, d, lap.shift, "d")
    assert not bench._unit_laplacian(bad)[0]
