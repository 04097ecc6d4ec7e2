"""Conjugate orthogonal CG for the shifted systems (oracle).

Algorithms 1 and 2 solve (z_j I - A) X_j = Q for every quadrature node; the
paper does not name the inner solver. Reading: COCG (van der Vorst and
Melissen, IEEE Trans. Magn. 26, 1990), the CG recurrence with the
unconjugated bilinear form x^T y, which is the natural Krylov solver for the
complex symmetric matrix z I - A (A real symmetric, z complex).

Per right-hand side b (each column independently):

    x0 = 0, r0 = b, p0 = r0, rho0 = r0^T r0
    repeat:
        w   = (z I - A) p
        mu  = p^T w                       (breakdown if |mu| <= 1e-30 |p| |w|)
        alpha = rho / mu
        x  += alpha p
        r  -= alpha w
        stop when ||r||_2 <= tol * ||b||_2 (Hermitian norm) or k = maxit
        rho' = r^T r,  beta = rho' / rho,  p = r + beta p

Columns are independent; they are processed side by side only so that numpy
does the arithmetic, each with its own scalars. A column whose right-hand
side is zero is converged at iteration 0 with x = 0.
"""
from __future__ import annotations

import dataclasses

import numpy as np


class CocgBreakdown(RuntimeError):
    pass


@dataclasses.dataclass
class CocgResult:
    x: np.ndarray          # complex [n, k]
    iters: np.ndarray      # int [k], iterations taken per column
    converged: np.ndarray  # bool [k]
    relres: np.ndarray     # final ||r|| / ||b|| per column (recursive r)


def bdot(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Unconjugated column-wise bilinear form u^T v."""
    return np.sum(u * v, axis=0)


def cocg(a_mul, z: complex, b: np.ndarray, tol: float, maxit: int) -> CocgResult:
    """Solve (z I - A) x = b column by column; ``a_mul(X)`` returns A @ X."""
    b = np.asarray(b, dtype=np.complex128)
    if b.ndim == 1:
        b = b[:, None]
    n, k = b.shape
    x = np.zeros((n, k), dtype=np.complex128)
    r = b.copy()
    p = r.copy()
    rho = bdot(r, r)
    bnorm = np.linalg.norm(b, axis=0)
    active = bnorm > 0.0
    converged = ~active
    iters = np.zeros(k, dtype=np.int64)
    relres = np.zeros(k)
    for _ in range(maxit):
        if not active.any():
            break
        w = z * p - a_mul(p)
        mu = bdot(p, w)
        pn = np.linalg.norm(p, axis=0)
        wn = np.linalg.norm(w, axis=0)
        bad = active & (np.abs(mu) <= 1e-30 * pn * wn)
        if bad.any():
            raise CocgBreakdown(f"COCG breakdown in columns {np.nonzero(bad)[0]}")
        alpha = np.where(active, rho / np.where(active, mu, 1.0), 0.0)
        x += alpha * p
        r -= alpha * w
        iters += active
        rn = np.linalg.norm(r, axis=0)
        done = active & (rn <= tol * bnorm)
        converged |= done
        active &= ~done
        rho_new = bdot(r, r)
        beta = np.where(active, rho_new / np.where(active, rho, 1.0), 0.0)
        rho = np.where(active, rho_new, rho)
        p = np.where(active, r + beta * p, p)
    rn = np.linalg.norm(r, axis=0)
    relres = np.where(bnorm > 0, rn / np.where(bnorm > 0, bnorm, 1.0), 0.0)
    return CocgResult(x=x, iters=iters, converged=converged, relres=relres)
