"""Pins of the oracle's exact-spectrum helpers and error metrics.

The closed forms (path, cycle, grid) are checked against brute-force dense
eigendecomposition of the generated Laplacians, ARPACK shift-invert against
dense eigh, and the trace identity trace(L) = sum of degrees.
"""
import numpy as np
import pytest

from oracle import exact as E
from oracle import metrics as M
from workloads import graphs as G


@pytest.mark.parametrize("n", [2, 7, 40])
def test_path_closed_form(n):
    lam = np.linalg.eigvalsh(G.path(n).scipy().toarray())
    assert np.allclose(np.sort(E.path_eigenvalues(n)), lam, atol=1e-12)
    for k in [0, 1, n - 1]:
        v = E.path_eigenvector(n, k)
        a = G.path(n).scipy()
        assert np.allclose(a @ v, E.path_eigenvalues(n)[k] * v, atol=1e-12)


@pytest.mark.parametrize("n", [3, 8, 31])
def test_cycle_closed_form(n):
    lam = np.linalg.eigvalsh(G.cycle(n).scipy().toarray())
    assert np.allclose(np.sort(E.cycle_eigenvalues(n)), lam, atol=1e-12)


@pytest.mark.parametrize("dims,shift", [((6, 5), 0.0), ((4, 3, 5), 0.01)])
def test_grid_closed_form(dims, shift):
    lap = G.grid2d(*dims, shift) if len(dims) == 2 else G.grid3d(*dims, shift)
    a = lap.scipy()
    lam = np.linalg.eigvalsh(a.toarray())
    vals, idx = E.grid_spectrum(dims, shift)
    assert np.allclose(vals, lam, atol=1e-12)
    for t in [0, 1, 5, len(vals) - 1]:
        v = E.grid_eigenvector(dims, idx[t])
        assert np.allclose(a @ v, vals[t] * v, atol=1e-12)
    assert abs(lam.sum() - (lap.values[lap.values > 0].sum() + shift * lap.n)) < 1e-9


def test_grid2d_40x50_interval():
    # the plain-FEAST workload: 16 eigenvalues in [0.0019733, 0.0792439]
    vals, _ = E.grid_spectrum((40, 50))
    assert E.count_in(vals, 0.0019733, 0.0792439) == 16
    assert abs(vals[1] - 0.003947) < 1e-6 and abs(vals[17] - 0.0874570) < 1e-6


def test_grid3d_100_interval():
    vals, _ = E.grid_spectrum((100, 100, 100), 0.01)
    assert E.count_in(vals, 0.005, 0.0272568) == 63
    inside = vals[vals <= 0.0272568]
    outside = vals[vals > 0.0272568]
    assert 0.0272568 - inside.max() > 4e-4 and outside.min() - 0.0272568 > 4e-4


def test_eigsh_matches_dense():
    lap = G.knn3d(600, 6, seed=5, shift=1e-3)
    a = lap.scipy()
    w, v = E.eigsh_smallest(a, 12)
    lam = np.linalg.eigvalsh(a.toarray())
    assert np.allclose(w, lam[:12], rtol=1e-11, atol=1e-13)
    assert np.linalg.norm(a @ v - v * w) < 1e-10


def test_lanczos_matches_dense_on_sbm():
    # a small stochastic block model: no geometric structure, the case the
    # factorisation-free Lanczos routine serves; brute force decides
    lap = G.sbm([120, 100, 130, 110], 20.0 / 115, 1.0 / 460, seed=9, shift=1e-3)
    a = lap.scipy()
    w, v = E.eigsh_smallest_lanczos(a, 12)
    lam = np.linalg.eigvalsh(a.toarray())
    assert np.allclose(w, lam[:12], rtol=1e-10, atol=1e-12)
    assert np.linalg.norm(a @ v - v * w) < 1e-9
    # the constant vector is the shifted Laplacian's eigenvector 1e-3
    assert abs(w[0] - 1e-3) < 1e-12


def test_sin_theta_metric():
    rng = np.random.default_rng(0)
    u, _ = np.linalg.qr(rng.standard_normal((50, 4)))
    assert M.sin_theta(u, u) < 1e-14
    # rotate the first column by a small angle out of the span
    perp = rng.standard_normal(50)
    perp -= u @ (u.T @ perp)
    perp /= np.linalg.norm(perp)
    for phi in [1e-12, 1e-6, 0.3]:
        v = u.copy()
        v[:, 0] = np.cos(phi) * u[:, 0] + np.sin(phi) * perp
        assert abs(M.sin_theta(v, u) - np.sin(phi)) < 1e-15 + 1e-9 * np.sin(phi)
    # a different basis of the same span has distance 0
    rot, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    assert M.sin_theta(u @ rot, u) < 1e-14


def test_eig_errors_and_orth():
    assert M.eig_relerr([1.0, 2.0], [2.0, 1.0]) == 0.0
    assert abs(M.eig_relerr([1.0 + 1e-9], [1.0]) - 1e-9) < 1e-15
    assert M.eig_relerr([1.0], [1.0, 2.0]) == float("inf")
    assert abs(M.eig_abserr([3.0], [2.5]) - 0.5) < 1e-15
    assert M.orth_err(np.eye(5)[:, :3]) == 0.0
