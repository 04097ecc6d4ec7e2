"""Pins of the oracle's COCG inner solver (shifted solves of Algorithm 1).

* dense direct solve of the complex symmetric system (numpy.linalg.solve);
* for a real shift below the spectrum, -(z I - A) is SPD and COCG is CG:
  its iterates must equal scipy's CG iterates step by step (callback);
* a zero right-hand side converges at iteration 0; a planted breakdown
  (p^T (zI - A) p = 0 at the first step) raises.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle import cocg as C


def _spd(n, seed, density=0.05):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng)
    m = m + m.T
    d = np.asarray(abs(m).sum(axis=1)).ravel() + 0.5
    return (m + sp.diags(d)).tocsr()


@pytest.mark.parametrize("z", [0.7 + 0.3j, 2.0 + 0.05j, -1.0 + 1.0j])
def test_matches_dense_solve(z):
    a = _spd(120, 0)
    rng = np.random.default_rng(1)
    b = rng.standard_normal((120, 3)) + 1j * rng.standard_normal((120, 3))
    res = C.cocg(lambda x: a @ x, z, b, 1e-13, 5000)
    assert res.converged.all()
    x = np.linalg.solve(z * np.eye(120) - a.toarray(), b)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-10


def test_real_shift_equals_cg_iterates():
    a = _spd(80, 2)
    lmin = np.linalg.eigvalsh(a.toarray()).min()
    z = lmin - 0.3
    rng = np.random.default_rng(3)
    b = rng.standard_normal(80)
    m = (a - z * sp.identity(80)).tocsr()  # SPD
    its = []
    sla.cg(m, -b, rtol=1e-300, atol=0.0, maxiter=12, callback=lambda xk: its.append(xk.copy()))
    for k in range(1, 12):
        res = C.cocg(lambda x: a @ x, complex(z), b, 0.0, k)
        assert np.allclose(res.x[:, 0].real, its[k - 1], rtol=1e-9, atol=1e-12)
        assert np.allclose(res.x[:, 0].imag, 0.0)


def test_zero_rhs_column():
    a = _spd(30, 4)
    b = np.zeros((30, 2))
    b[:, 1] = 1.0
    res = C.cocg(lambda x: a @ x, 1.0 + 1.0j, b, 1e-12, 500)
    assert res.iters[0] == 0 and res.converged[0]
    assert np.all(res.x[:, 0] == 0)
    assert res.converged[1] and res.iters[1] > 0


def test_planted_breakdown_raises():
    # z I - A = diag(1, -1) (A = diag(-1, 1), z = 0) and b = (1, 1):
    # b^T (zI - A) b = 0, so the first mu vanishes.
    a = sp.diags([-1.0, 1.0]).tocsr()
    with pytest.raises(C.CocgBreakdown):
        C.cocg(lambda x: a @ x, 0.0 + 0.0j, np.array([1.0, 1.0]), 1e-12, 10)


def test_iteration_cap():
    a = _spd(200, 5)
    b = np.ones(200)
    res = C.cocg(lambda x: a @ x, 1.0 + 1e-3j, b, 1e-14, 3)
    assert res.iters[0] == 3 and not res.converged[0]


def test_bdot_is_unconjugated():
    # u^T v without conjugation: (1 + 2i) * (3 - i) + 1j * 1j = 5 + 5i - 1
    u = np.array([[1 + 2j], [1j]])
    v = np.array([[3 - 1j], [1j]])
    assert np.allclose(C.bdot(u, v), [4 + 5j])
    # column by column
    u2 = np.hstack([u, 2 * u])
    v2 = np.hstack([v, v])
    assert np.allclose(C.bdot(u2, v2), [4 + 5j, 8 + 10j])
