"""FEAST and RA-FEAST outer loops in FP64 (oracle).

Follows Algorithm 1 (FEAST iteration) and Algorithm 2 (RA-FEAST) step by
step; the readings of what the paper leaves open are stated where they are
used:

* Filter (Algorithm 1 step "Compute Q~"; Algorithm 2 Step 2a): for every
  node solve (z_j I - A) X_j = Q, then Q~ = sum_j Re(w_j X_j). The real part
  is taken because the lower half of the contour is the conjugate of the
  upper half (see ``quadrature``).
* The solve may be written in *correction form*. For any real scalar theta
  per column, (z I - A)^{-1} q = q/(z - theta)
  + (z I - A)^{-1} (A q - theta q) / (z - theta), an algebraic identity, so
  both forms compute the same X_j; they differ only in how an inexact inner
  solve errs. With theta the Rayleigh quotient, the inner solve's error then
  scales with the current residual instead of with ||q||, which lets a
  relaxed inner tolerance (Section 3.1, Phase 2) still reach a tight outer
  tolerance (Theorem 2: the perturbation eps^(m) shrinks with the residual).
* Orthonormalise Q^(m+1) R = Q~ with Householder QR (numpy.linalg.qr).
* Rayleigh-Ritz: A_Q = Q^T A Q = V L V^T (ascending), Q <- Q V.
* Convergence (the paper says only "until convergence"): relative residual
  ||A q_i - l_i q_i||_2 / ||A||_1 of every Ritz pair inside the interval is
  at most ``outer_tol``; also stop at ``max_outer``.
* Warmstart (Algorithm 2 Phase 1): B is an affine map of A under which the
  target interval becomes the dominant part of the spectrum. The paper's
  literal B = (A - lmin I)/(lmax - lmin) does that only for an interval at the
  top of the spectrum; for an interval in the lower half the map
  B = (g I - A)/(g - lmin), g the Gershgorin upper bound, plays the same role
  (Assumption 1.2's "appropriate transformation", kept polynomial).
  Y = (B B^T)^q B Omega = B^{2q+1} Omega, re-orthonormalised after each pair of
  products (only the basis changes), Q0 = orth(Y), then Rayleigh-Ritz on A
  keeps the m0 Ritz vectors whose Ritz values are closest to the interval
  centre (Omega has m0+p columns, the FEAST subspace m0).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import cocg as _cocg
from . import philox as _philox
from . import quadrature as _quad

STATUS_OK = 0
STATUS_NO_EIGENVALUE = 1
STATUS_NO_CONVERGENCE = 2
STATUS_M0_TOO_SMALL = 3


def one_norm(a: sp.spmatrix) -> float:
    """||A||_1 = max column sum of |a_ij|."""
    return float(np.max(np.asarray(abs(a).sum(axis=0)).ravel()))


def gershgorin(a: sp.spmatrix):
    """(lower, upper) Gershgorin bounds of a real symmetric matrix."""
    a = sp.csr_matrix(a)
    d = a.diagonal()
    off = np.asarray(abs(a).sum(axis=1)).ravel() - np.abs(d)
    return float(np.min(d - off)), float(np.max(d + off))


def filter_apply(a: sp.spmatrix, q: np.ndarray, z, w, solve_tol: float,
                 max_inner: int, form: str = "direct",
                 theta: np.ndarray | None = None):
    """Q~ = sum_j Re(w_j X_j) with (z_j I - A) X_j = Q (Algorithm 1/2).

    ``form='direct'`` hands Q to COCG; ``form='correction'`` hands it the
    residual R = A Q - Q diag(theta) and rebuilds X_j = (Q + Y_j) / (z_j -
    theta), Y_j solving (z_j I - A) Y_j = R. ``theta`` defaults to the
    Rayleigh quotients of the columns of Q. Returns (Q~, list of COCG
    results per node)."""
    a = sp.csr_matrix(a)
    amul = lambda x: a @ x  # noqa: E731
    q = np.asarray(q, dtype=np.float64)
    qt = np.zeros_like(q)
    stats = []
    if form == "direct":
        for zj, wj in zip(z, w):
            res = _cocg.cocg(amul, zj, q, solve_tol, max_inner)
            stats.append(res)
            qt += np.real(wj * res.x)
    elif form == "correction":
        aq = a @ q
        if theta is None:
            theta = np.sum(q * aq, axis=0) / np.sum(q * q, axis=0)
        rmat = aq - q * theta
        for zj, wj in zip(z, w):
            res = _cocg.cocg(amul, zj, rmat, solve_tol, max_inner)
            stats.append(res)
            xj = (q + res.x) / (zj - theta)
            qt += np.real(wj * xj)
    else:
        raise ValueError(form)
    return qt, stats


def orthonormalize(qt: np.ndarray) -> np.ndarray:
    """Q R = Q~ (Householder QR); returns Q."""
    q, _ = np.linalg.qr(qt)
    return q


def rayleigh_ritz(a: sp.spmatrix, q: np.ndarray):
    """A_Q = Q^T A Q = V L V^T; returns (L ascending, Q V, A Q V)."""
    aq = a @ q
    aqq = q.T @ aq
    aqq = 0.5 * (aqq + aqq.T)
    lam, v = np.linalg.eigh(aqq)
    return lam, q @ v, aq @ v


def residuals(a: sp.spmatrix, lam: np.ndarray, q: np.ndarray,
              aq: np.ndarray | None = None, norm_a: float | None = None):
    """||A q_i - lam_i q_i||_2 / ||A||_1 per column."""
    if aq is None:
        aq = a @ q
    if norm_a is None:
        norm_a = one_norm(a)
    return np.linalg.norm(aq - q * lam, axis=0) / norm_a


def random_start(n: int, m0: int, seed: int) -> np.ndarray:
    """Algorithm 1 initial subspace: orthonormalised Gaussian block drawn
    with the same Philox-4x64-10 generator as Omega."""
    return orthonormalize(_philox.gaussian_matrix(n, m0, seed))


@dataclasses.dataclass
class FeastResult:
    status: int
    evals: np.ndarray        # in-interval Ritz values, ascending
    evecs: np.ndarray        # [n, m_found]
    resid: np.ndarray        # [m_found]
    m_found: int
    outer_iters: int
    ritz_all: np.ndarray     # all m0 Ritz values of the last iterate
    q_all: np.ndarray        # all m0 Ritz vectors of the last iterate
    res_all: np.ndarray
    history: list            # per outer iteration: dict of diagnostics


def feast(a: sp.spmatrix, lmin: float, lmax: float, q0: np.ndarray, nc: int,
          e: float = 1.0, solve_tol: float = 1e-10, outer_tol: float = 1e-10,
          max_outer: int = 20, max_inner: int = 10000, form: str = "direct",
          theta0: np.ndarray | None = None) -> FeastResult:
    """FEAST outer loop (Algorithm 1, and Phase 2 of Algorithm 2).

    Each iteration: filter (all N_c shifted solves), QR, Rayleigh-Ritz,
    residuals, convergence test on the Ritz pairs inside [lmin, lmax]."""
    a = sp.csr_matrix(a)
    z, w = _quad.nodes(lmin, lmax, nc, e)
    norm_a = one_norm(a)
    q = np.asarray(q0, dtype=np.float64)
    m0 = q.shape[1]
    theta = theta0
    history = []
    status = STATUS_NO_CONVERGENCE
    lam = res = None
    it = 0
    for it in range(1, max_outer + 1):
        qt, stats = filter_apply(a, q, z, w, solve_tol, max_inner, form, theta)
        q = orthonormalize(qt)
        lam, q, aq = rayleigh_ritz(a, q)
        theta = lam
        res = residuals(a, lam, q, aq, norm_a)
        inside = (lam >= lmin) & (lam <= lmax)
        iters = np.concatenate([s.iters for s in stats])
        history.append(dict(m=it, n_inside=int(inside.sum()),
                            max_res=float(res[inside].max()) if inside.any() else np.nan,
                            cocg_min=int(iters.min()), cocg_max=int(iters.max())))
        if inside.any() and res[inside].max() <= outer_tol:
            status = STATUS_OK
            break
    inside = (lam >= lmin) & (lam <= lmax)
    mf = int(inside.sum())
    if mf == 0:
        status = STATUS_NO_EIGENVALUE
    elif mf >= m0:
        # every Ritz value inside: the interval may hold m0 or more
        # eigenvalues, so "none missed" cannot be claimed, converged or not
        status = STATUS_M0_TOO_SMALL
    return FeastResult(status=status, evals=lam[inside], evecs=q[:, inside],
                       resid=res[inside], m_found=mf, outer_iters=it,
                       ritz_all=lam, q_all=q, res_all=res, history=history)


def warmstart_map(a: sp.spmatrix, lmin: float, lmax: float,
                  which: str = "auto"):
    """Affine map B = s A + t I of the warmstart (Algorithm 2 Phase 1),
    returned as (s, t, name). ``which='literal'`` is the paper's
    (A - lmin I)/(lmax - lmin); ``'low'`` is (g I - A)/(g - lmin) with g the
    Gershgorin upper bound; ``'auto'`` picks ``'literal'`` when the interval
    centre lies in the upper half of the Gershgorin range, else ``'low'``."""
    glo, ghi = gershgorin(a)
    if which == "auto":
        which = "literal" if 0.5 * (lmin + lmax) >= 0.5 * (glo + ghi) else "low"
    if which == "literal":
        s = 1.0 / (lmax - lmin)
        return s, -lmin * s, "literal"
    if which == "low":
        s = -1.0 / (ghi - lmin)
        return s, ghi / (ghi - lmin), "low"
    raise ValueError(which)


def warmstart(a: sp.spmatrix, lmin: float, lmax: float, m0: int, p: int,
              q: int, omega: np.ndarray, which: str = "auto"):
    """Randomized warmstart (Algorithm 2 Phase 1, Eq. 6 applied to B).

    Returns (Q0 [n, m0], Ritz values of Q0 [m0], details dict)."""
    a = sp.csr_matrix(a)
    s, t, name = warmstart_map(a, lmin, lmax, which)
    bmul = lambda x: s * (a @ x) + t * x  # noqa: E731
    y = bmul(np.asarray(omega, dtype=np.float64))
    for _ in range(q):
        y = orthonormalize(y)
        y = bmul(bmul(y))
    qw = orthonormalize(y)
    lam, qv, _ = rayleigh_ritz(a, qw)
    c = 0.5 * (lmin + lmax)
    order = np.argsort(np.abs(lam - c), kind="stable")[:m0]
    keep = np.sort(order)
    return qv[:, keep], lam[keep], dict(map=name, s=s, t=t, ritz_all=lam)


def rafeast(a: sp.spmatrix, lmin: float, lmax: float, m0: int, p: int, q: int,
            seed: int, nc: int, e: float = 1.0, solve_tol: float = 1e-4,
            outer_tol: float = 1e-10, max_outer: int = 20,
            max_inner: int = 10000, form: str = "correction",
            which: str = "auto") -> FeastResult:
    """RA-FEAST (Algorithm 2): Phase 1 warmstart, Phase 2 FEAST."""
    n = a.shape[0]
    omega = _philox.gaussian_matrix(n, m0 + p, seed)
    q0, theta0, _ = warmstart(a, lmin, lmax, m0, p, q, omega, which)
    return feast(a, lmin, lmax, q0, nc, e, solve_tol, outer_tol, max_outer,
                 max_inner, form, theta0)
