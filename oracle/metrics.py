"""Error measures between computed and reference eigenpairs (oracle).

* ``sin_theta(U, V)``: ||U - V (V^T U)||_2 for orthonormal U, V, the 2-norm of
  the sine of the canonical angles (Lemma 2, Eq. 11: ||P - P~||_2 =
  ||sin Theta||_2). Written as a residual projection rather than
  sqrt(1 - sigma_min(V^T U)^2), which loses every digit below ~1e-8.
  Eigenvectors of repeated eigenvalues are not unique, so comparing whole
  subspaces is what is meaningful.
* ``eig_relerr``: max_i |l^_i - l_i| / |l_i| over matched (sorted) lists;
  ``eig_abserr`` is the paper's Table 1 metric max_i |l^_i - l_i|.
* ``orth_err``: ||Q^T Q - I||_F.
"""
from __future__ import annotations

import numpy as np


def sin_theta(u: np.ndarray, v: np.ndarray) -> float:
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    if u.shape[1] == 0 and v.shape[1] == 0:
        return 0.0
    return float(np.linalg.norm(u - v @ (v.T @ u), 2))


def eig_relerr(got, ref) -> float:
    got = np.sort(np.asarray(got, dtype=np.float64))
    ref = np.sort(np.asarray(ref, dtype=np.float64))
    if got.shape != ref.shape:
        return float("inf")
    if got.size == 0:
        return 0.0
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def eig_abserr(got, ref) -> float:
    got = np.sort(np.asarray(got, dtype=np.float64))
    ref = np.sort(np.asarray(ref, dtype=np.float64))
    if got.shape != ref.shape:
        return float("inf")
    if got.size == 0:
        return 0.0
    return float(np.max(np.abs(got - ref)))


def orth_err(q: np.ndarray) -> float:
    q = np.asarray(q, dtype=np.float64)
    return float(np.linalg.norm(q.T @ q - np.eye(q.shape[1])))
