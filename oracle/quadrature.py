"""Contour quadrature for the FEAST spectral projector (oracle).

Section 2.1, Eq. 2 (projector as a contour integral of the resolvent) and
Eq. 3 (its N_c-point quadrature). The paper does not fix the rule or the
contour. Reading used here: Gauss-Legendre on the upper half of an ellipse
centred at c = (lmin+lmax)/2 with real semi-axis R = (lmax-lmin)/2 and
imaginary semi-axis e*R. Because A is real symmetric, the lower half of the
contour contributes the complex conjugate of the upper half, so the
projector is 2*Re of the upper-half sum; the factor 2 and the orientation are
folded into w_j below and the caller takes the real part of
sum_j w_j (z_j I - A)^{-1}.

Parametrise z(t) = c + R cos t + i e R sin t, t in [0, pi]. With GL points
x_j and weights om_j on [-1, 1] and t_j = (pi/2)(1 + x_j),

    z_j = c + R (cos t_j + i e sin t_j)
    w_j = (R om_j / 2) (e cos t_j + i sin t_j)

and the scalar filter of the quadrature is f(l) = sum_j Re(w_j / (z_j - l)).
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(nc: int):
    """GL points and weights on [-1, 1] (library routine)."""
    x, om = np.polynomial.legendre.leggauss(nc)
    return x, om


def nodes(lmin: float, lmax: float, nc: int, e: float = 1.0):
    """Quadrature nodes z_j and weights w_j, j = 1..nc (Eq. 3)."""
    if not lmax > lmin:
        raise ValueError("need lmin < lmax")
    if nc < 1:
        raise ValueError("need nc >= 1")
    if not (0.0 < e <= 1.0):
        raise ValueError("ellipse ratio must lie in (0, 1]")
    x, om = gauss_legendre(nc)
    c = 0.5 * (lmin + lmax)
    r = 0.5 * (lmax - lmin)
    t = 0.5 * np.pi * (1.0 + x)
    z = c + r * (np.cos(t) + 1j * e * np.sin(t))
    w = 0.5 * r * om * (e * np.cos(t) + 1j * np.sin(t))
    return z.astype(np.complex128), w.astype(np.complex128)


def filter_value(lam, z, w):
    """Rational filter f(lam) = sum_j Re(w_j / (z_j - lam)): the scalar the
    quadrature projector applies to an eigenvector with eigenvalue lam."""
    lam = np.asarray(lam, dtype=np.float64)
    out = np.zeros(lam.shape, dtype=np.float64)
    for zj, wj in zip(z, w):
        out += np.real(wj / (zj - lam))
    return out
