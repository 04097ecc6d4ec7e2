"""Seeded synthetic sparse graph Laplacians.

This module only builds input matrices. It holds none of the eigensolver's
arithmetic and is shared by the CPU oracle, the tests and the benchmark.

Every generator returns a ``Laplacian``: the exact graph Laplacian L = D - W
in CSR form (int32 indices, float64 values that are small integers for the
unit-weight graphs used here) plus a scalar ``shift`` so that the SPD matrix
studied is A = L + shift * I. Keeping the shift outside the CSR keeps the
integer Laplacian values exact when they are later rounded to float32.

Workload families (all unit-weight, undirected, no self loops):

* ``grid2d(nx, ny)``: 5-point grid graph (Cartesian product of two paths).
* ``grid3d(nx, ny, nz)``: 7-point grid graph (product of three paths).
* ``knn3d(n, k, seed)``: k nearest neighbours of n uniform points in the unit
  cube, symmetrised by union (edge if either endpoint lists the other).
* ``sbm(sizes, p_in, p_out, seed)``: stochastic block model.
* ``rgg2d(n, radius, seed)``: random geometric graph in the unit square, the
  graph family of the paper's experiments (Section 5.1).
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Laplacian:
    """CSR graph Laplacian plus a scalar diagonal shift (A = L + shift*I)."""

    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col_idx: np.ndarray  # int32 [nnz], sorted within each row
    values: np.ndarray   # float64 [nnz]
    shift: float
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def scipy(self, with_shift: bool = True) -> sp.csr_matrix:
        """The matrix as scipy CSR (A when ``with_shift``, else L)."""
        m = sp.csr_matrix((self.values, self.col_idx, self.row_ptr),
                          shape=(self.n, self.n))
        if with_shift and self.shift != 0.0:
            m = (m + self.shift * sp.identity(self.n, format="csr")).tocsr()
            m.sort_indices()
        return m

    def checksum(self) -> str:
        """Digest of the CSR arrays, used to assert that a stored expected
        value refers to the same matrix on every machine."""
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(self.row_ptr, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(self.col_idx, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(self.values, dtype=np.float64).tobytes())
        h.update(np.float64(self.shift).tobytes())
        return h.hexdigest()[:16]


def _from_edges(n: int, i: np.ndarray, j: np.ndarray, shift: float,
                name: str) -> Laplacian:
    """Unit-weight Laplacian from an undirected edge list (i < j, unique)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    rows = np.concatenate([i, j])
    cols = np.concatenate([j, i])
    w = sp.csr_matrix((np.ones(rows.shape[0]), (rows, cols)), shape=(n, n))
    w.sum_duplicates()
    w.data[:] = 1.0
    deg = np.asarray(w.sum(axis=1)).ravel()
    lap = (sp.diags(deg) - w).tocsr()
    lap.sum_duplicates()
    lap.sort_indices()
    lap.eliminate_zeros()   # an isolated vertex keeps an empty CSR row
    return Laplacian(n=n,
                     row_ptr=lap.indptr.astype(np.int32),
                     col_idx=lap.indices.astype(np.int32),
                     values=lap.data.astype(np.float64),
                     shift=float(shift), name=name)


def path_edges(n: int):
    i = np.arange(n - 1)
    return i, i + 1


def grid2d(nx: int, ny: int, shift: float = 0.0) -> Laplacian:
    """5-point grid graph; vertex (a, b) has index a + nx*b."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    ei = [idx[:, :-1].ravel(), idx[:-1, :].ravel()]
    ej = [idx[:, 1:].ravel(), idx[1:, :].ravel()]
    return _from_edges(nx * ny, np.concatenate(ei), np.concatenate(ej), shift,
                       f"grid2d_{nx}x{ny}")


def grid3d(nx: int, ny: int, nz: int, shift: float = 0.0) -> Laplacian:
    """7-point grid graph; vertex (a, b, c) has index a + nx*(b + ny*c)."""
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    ei = [idx[:, :, :-1].ravel(), idx[:, :-1, :].ravel(), idx[:-1, :, :].ravel()]
    ej = [idx[:, :, 1:].ravel(), idx[:, 1:, :].ravel(), idx[1:, :, :].ravel()]
    return _from_edges(nx * ny * nz, np.concatenate(ei), np.concatenate(ej),
                       shift, f"grid3d_{nx}x{ny}x{nz}")


def path(n: int, shift: float = 0.0) -> Laplacian:
    i, j = path_edges(n)
    return _from_edges(n, i, j, shift, f"path_{n}")


def cycle(n: int, shift: float = 0.0) -> Laplacian:
    i, j = path_edges(n)
    i = np.append(i, 0)
    j = np.append(j, n - 1)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    return _from_edges(n, lo, hi, shift, f"cycle_{n}")


def knn3d(n: int, k: int = 10, seed: int = 1, shift: float = 1e-3) -> Laplacian:
    """kNN graph of n points drawn uniformly in [0,1]^3 with
    ``numpy.random.default_rng(seed)``; union-symmetrised, unit weights."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    tree = cKDTree(pts)
    _, nbr = tree.query(pts, k=k + 1)
    src = np.repeat(np.arange(n), k)
    dst = nbr[:, 1:].ravel()
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    keep = lo != hi
    key = np.unique(lo[keep].astype(np.int64) * n + hi[keep])
    return _from_edges(n, key // n, key % n, shift, f"knn3d_n{n}_k{k}_s{seed}")


def rgg2d(n: int, radius: float | None = None, seed: int = 0,
          shift: float = 0.0) -> Laplacian:
    """Random geometric graph: n uniform points in [0,1]^2, edge when the
    distance is below ``radius`` (default 1.5*sqrt(log(n)/n), Section 5.1)."""
    from scipy.spatial import cKDTree

    if radius is None:
        radius = 1.5 * np.sqrt(np.log(n) / n)
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    pairs = cKDTree(pts).query_pairs(radius, output_type="ndarray")
    return _from_edges(n, pairs[:, 0], pairs[:, 1], shift, f"rgg2d_n{n}_s{seed}")


def sbm(sizes, p_in: float, p_out: float, seed: int,
        shift: float = 1e-3) -> Laplacian:
    """Stochastic block model with contiguous blocks.

    For every block pair the edge count is drawn from the binomial law of the
    model, then that many vertex pairs are drawn uniformly (with replacement)
    and duplicates are merged: O(edges) work, never O(n^2).
    """
    rng = np.random.default_rng(seed)
    sizes = [int(s) for s in sizes]
    starts = np.concatenate([[0], np.cumsum(sizes)])
    n = int(starts[-1])
    chunks_i, chunks_j = [], []
    nb = len(sizes)
    for a in range(nb):
        for b in range(a, nb):
            na, nbb = sizes[a], sizes[b]
            if a == b:
                pairs = na * (na - 1) // 2
                p = p_in
            else:
                pairs = na * nbb
                p = p_out
            if pairs == 0 or p <= 0:
                continue
            m = int(rng.binomial(pairs, min(p, 1.0)))
            if m == 0:
                continue
            i = starts[a] + rng.integers(0, na, size=m)
            j = starts[b] + rng.integers(0, nbb, size=m)
            chunks_i.append(i)
            chunks_j.append(j)
    i = np.concatenate(chunks_i)
    j = np.concatenate(chunks_j)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    keep = lo != hi
    key = np.unique(lo[keep].astype(np.int64) * n + hi[keep])
    return _from_edges(n, key // n, key % n, shift,
                       f"sbm_n{n}_K{nb}_s{seed}")
