"""Pins of the oracle's contour quadrature (Section 2.1, Eq. 2-3).

The filter f(l) = sum_j Re(w_j/(z_j - l)) is fixed by mathematics in several
places, none of which re-types the node formula:

* circle (e = 1): z_j - c = R e^{i t_j} and w_j = (R om_j/2) e^{i t_j}, so
  f(c) = sum_j om_j / 2 = 1 (Gauss-Legendre weights sum to 2);
* circle, at the interval ends: e^{it}/(e^{it} - 1) = 1/2 - (i/2) cot(t/2)
  has real part 1/2 for every t, so f(lmin) = f(lmax) = 1/2 exactly;
* N_c = 1: one node at t = pi/2, z = c + i e R, w = i R, hence
  f(l) = e R^2 / ((c - l)^2 + e^2 R^2), a Lorentzian;
* the nodes are symmetric under t -> pi - t, so f(c + s) = f(c - s);
* as N_c grows, f tends to the indicator of the interval (the exact
  projector of Eq. 2 maps each eigenvector to itself inside, to 0 outside).
"""
import numpy as np
import pytest

from oracle import quadrature as Q


@pytest.mark.parametrize("nc", [1, 2, 3, 4, 8, 16])
def test_circle_centre_and_ends(nc):
    lmin, lmax = 0.3, 1.7
    z, w = Q.nodes(lmin, lmax, nc, 1.0)
    c = 0.5 * (lmin + lmax)
    assert abs(Q.filter_value(c, z, w) - 1.0) < 1e-14
    assert abs(Q.filter_value(lmin, z, w) - 0.5) < 1e-13
    assert abs(Q.filter_value(lmax, z, w) - 0.5) < 1e-13


@pytest.mark.parametrize("e", [1.0, 0.5, 0.3])
def test_single_node_lorentzian(e):
    lmin, lmax = -1.0, 3.0
    c, r = 1.0, 2.0
    z, w = Q.nodes(lmin, lmax, 1, e)
    lam = np.linspace(-5, 7, 41)
    expect = e * r * r / ((c - lam) ** 2 + (e * r) ** 2)
    assert np.allclose(Q.filter_value(lam, z, w), expect, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("nc,e", [(2, 1.0), (4, 0.3), (8, 1.0), (5, 0.7)])
def test_symmetry_about_centre(nc, e):
    z, w = Q.nodes(2.0, 4.0, nc, e)
    s = np.linspace(0, 5, 23)
    assert np.allclose(Q.filter_value(3.0 + s, z, w),
                       Q.filter_value(3.0 - s, z, w), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("e", [1.0, 0.5])
def test_tends_to_indicator(e):
    lmin, lmax = 1.0, 2.0
    z, w = Q.nodes(lmin, lmax, 48, e)
    inside = np.linspace(1.2, 1.8, 13)
    outside = np.concatenate([np.linspace(-3, 0.8, 9), np.linspace(2.2, 9, 9)])
    assert np.all(np.abs(Q.filter_value(inside, z, w) - 1.0) < 1e-4)
    assert np.all(np.abs(Q.filter_value(outside, z, w)) < 1e-4)


def test_nodes_on_upper_half_ellipse():
    lmin, lmax, e = 0.0, 2.0, 0.4
    z, w = Q.nodes(lmin, lmax, 6, e)
    c, r = 1.0, 1.0
    assert np.all(z.imag > 0)
    assert np.allclose(((z.real - c) / r) ** 2 + (z.imag / (e * r)) ** 2, 1.0)


def test_contraction_matches_closed_form_for_nc2():
    # N_c = 2: x = +-1/sqrt(3), om = 1, t = (pi/2)(1 -+ 1/sqrt(3)).
    # Evaluate f from the contour sum written with these t (independent of
    # leggauss) at a few points.
    lmin, lmax = 0.0, 2.0
    c, r = 1.0, 1.0
    t = 0.5 * np.pi * (1.0 + np.array([-1.0, 1.0]) / np.sqrt(3.0))
    lam = np.array([-0.5, 0.25, 1.0, 2.5, 4.0])
    f = np.zeros_like(lam)
    for tj in t:
        zj = c + r * np.exp(1j * tj)
        wj = 0.5 * r * np.exp(1j * tj)
        f += np.real(wj / (zj - lam))
    z, w = Q.nodes(lmin, lmax, 2, 1.0)
    assert np.allclose(Q.filter_value(lam, z, w), f, rtol=1e-14)


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        Q.nodes(1.0, 1.0, 4)
    with pytest.raises(ValueError):
        Q.nodes(0.0, 1.0, 0)
    with pytest.raises(ValueError):
        Q.nodes(0.0, 1.0, 2, 1.5)


def test_gauss_legendre_three_point_rule():
    # the textbook 3-point rule: nodes 0, +-sqrt(3/5), weights 8/9, 5/9; it
    # integrates polynomials up to degree 5 exactly
    x, om = Q.gauss_legendre(3)
    order = np.argsort(x)
    assert np.allclose(x[order], [-np.sqrt(0.6), 0.0, np.sqrt(0.6)], atol=1e-15)
    assert np.allclose(om[order], [5 / 9, 8 / 9, 5 / 9], atol=1e-15)
    for deg in range(6):
        exact = (1.0 - (-1.0) ** (deg + 1)) / (deg + 1)
        assert abs(np.sum(om * x ** deg) - exact) <= 1e-14
