"""The exact answer FEAST converges to (oracle).

Eq. 1 defines the target: every eigenpair of A with eigenvalue in
[lmin, lmax]. This module computes it without FEAST:

* closed forms for path, cycle and grid graph Laplacians (the grid graph is
  a Cartesian product of paths, so its spectrum is the set of sums of path
  eigenvalues and its eigenvectors are products of path eigenvectors);
* dense ``numpy.linalg.eigh`` for small n;
* ARPACK (``scipy.sparse.linalg.eigsh``) in shift-invert mode about a real
  shift, with a SuperLU factorisation in a symmetric minimum-degree order,
  for large sparse A (ARPACK is the library behind the RSpectra ground truth
  of Section 5.1);
* ARPACK's implicitly restarted Lanczos on A itself (smallest algebraic
  eigenvalues, no factorisation) for sparse graphs without geometric
  structure, whose LU factors would fill in (stochastic block models).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def path_eigenvalues(n: int) -> np.ndarray:
    """Laplacian of the path P_n: 2 - 2 cos(pi k / n), k = 0..n-1."""
    k = np.arange(n)
    return 2.0 - 2.0 * np.cos(np.pi * k / n)


def path_eigenvector(n: int, k: int) -> np.ndarray:
    """Unit eigenvector cos(pi k (i + 1/2) / n) of the path Laplacian."""
    i = np.arange(n)
    v = np.cos(np.pi * k * (i + 0.5) / n)
    return v / np.linalg.norm(v)


def cycle_eigenvalues(n: int) -> np.ndarray:
    """Laplacian of the cycle C_n: 2 - 2 cos(2 pi k / n), k = 0..n-1."""
    k = np.arange(n)
    return 2.0 - 2.0 * np.cos(2.0 * np.pi * k / n)


def grid_spectrum(dims, shift: float = 0.0):
    """All eigenvalues of the grid graph Laplacian on ``dims`` (+ shift I),
    with their multi-indices; vertex (a, b, ...) has index
    a + d0*(b + d1*(...)). Returns (values ascending, index tuples)."""
    per = [path_eigenvalues(d) for d in dims]
    mesh = np.meshgrid(*per, indexing="ij")
    vals = sum(m.ravel() for m in mesh) + shift
    idx = np.array(list(itertools.product(*[range(d) for d in dims])))
    order = np.argsort(vals, kind="stable")
    return vals[order], idx[order]


def grid_eigenvector(dims, kidx) -> np.ndarray:
    """Product eigenvector for multi-index ``kidx`` (same vertex order as
    ``workloads.graphs.grid2d/grid3d``: first coordinate fastest)."""
    v = np.ones(1)
    for d, k in zip(dims, kidx):
        v = np.kron(path_eigenvector(d, k), v)
    return v


def grid_eigvecs_in(dims, shift: float, lmin: float, lmax: float):
    """Closed-form eigenpairs of the grid Laplacian in [lmin, lmax]."""
    vals, idx = grid_spectrum(dims, shift)
    sel = (vals >= lmin) & (vals <= lmax)
    vecs = np.stack([grid_eigenvector(dims, k) for k in idx[sel]], axis=1)
    return vals[sel], vecs


def dense_eigh(a) -> tuple[np.ndarray, np.ndarray]:
    """All eigenpairs by dense eigh (brute force, small n)."""
    if sp.issparse(a):
        a = a.toarray()
    return np.linalg.eigh(np.asarray(a, dtype=np.float64))


def eigsh_smallest(a: sp.spmatrix, k: int, sigma: float = 0.0,
                   tol: float = 1e-13):
    """k eigenpairs nearest ``sigma`` (from above, for sigma below the
    spectrum) by ARPACK shift-invert; returns ascending values, vectors."""
    a = sp.csc_matrix(a)
    n = a.shape[0]
    m = (a - sigma * sp.identity(n, format="csc")).tocsc()
    lu = sla.splu(m, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                  options=dict(SymmetricMode=True))
    op = sla.LinearOperator(a.shape, matvec=lu.solve, dtype=np.float64)
    w, v = sla.eigsh(a, k=k, sigma=sigma, which="LM", OPinv=op, tol=tol)
    order = np.argsort(w)
    return w[order], v[:, order]


def eigsh_smallest_lanczos(a: sp.spmatrix, k: int, tol: float = 1e-12,
                           seed: int = 0):
    """k smallest eigenpairs of the symmetric A by ARPACK Lanczos (which =
    'SA') with a seeded start vector; returns ascending values, vectors."""
    a = sp.csr_matrix(a)
    n = a.shape[0]
    v0 = np.random.default_rng(seed).standard_normal(n)
    ncv = min(n, max(4 * k, 60))
    w, v = sla.eigsh(a, k=k, which="SA", tol=tol, ncv=ncv, v0=v0)
    order = np.argsort(w)
    return w[order], v[:, order]


def count_in(vals: np.ndarray, lmin: float, lmax: float) -> int:
    return int(np.sum((vals >= lmin) & (vals <= lmax)))
