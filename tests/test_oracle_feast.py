"""Pins of the oracle's FEAST / RA-FEAST loops (Algorithms 1 and 2).

* Filter by solves equals the spectral-calculus operator V f(L) V^T applied
  to Q (dense eigendecomposition, a different route to the same operator),
  in both the direct and the correction form.
* Converged eigenpairs equal the closed-form grid spectrum / dense eigh
  (Eq. 1: every eigenpair inside the interval, none missed).
* Ritz values of any subspace lie above the true ones (Courant-Fischer).
* The observed outer contraction matches |f(l_(m0+1))| / min_inside |f| of
  subspace iteration with the filter operator (Theorem 2's rho for exact
  solves).
* Warmstart: the affine map sends lmin to 1 and the far end to 0; the
  range finder obeys Lemma 1 + Lemma 2's bound (Theorem 1).
* Status codes: empty interval, m0 too small, iteration cap.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import exact as E
from oracle import feast as F
from oracle import metrics as M
from oracle import philox as P
from oracle import quadrature as Q
from workloads import graphs as G


def _random_spd(n, seed):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=0.04, random_state=rng)
    m = (m + m.T) * 0.5
    d = np.asarray(abs(m).sum(axis=1)).ravel() + 0.05
    return (m + sp.diags(d)).tocsr()


@pytest.mark.parametrize("form", ["direct", "correction"])
@pytest.mark.parametrize("nc,e", [(2, 1.0), (4, 0.3), (8, 1.0)])
def test_filter_equals_spectral_calculus(form, nc, e):
    a = _random_spd(90, 0)
    lam, v = np.linalg.eigh(a.toarray())
    lmin, lmax = lam[3] - 1e-3, lam[12] + 1e-3
    z, w = Q.nodes(lmin, lmax, nc, e)
    q = F.random_start(90, 10, 7)
    qt, stats = F.filter_apply(a, q, z, w, 1e-14, 2000, form)
    expect = v @ (Q.filter_value(lam, z, w)[:, None] * (v.T @ q))
    assert np.linalg.norm(qt - expect) / np.linalg.norm(expect) < 1e-11
    assert all(s.converged.all() for s in stats)


def test_feast_grid_closed_form():
    dims = (12, 10)
    a = G.grid2d(*dims).scipy()
    vals, _ = E.grid_spectrum(dims)
    lmin = 0.5 * (vals[2] + vals[3])
    lmax = 0.5 * (vals[9] + vals[10])
    ref_vals, ref_vecs = E.grid_eigvecs_in(dims, 0.0, lmin, lmax)
    q0 = F.random_start(a.shape[0], 12, 1)
    r = F.feast(a, lmin, lmax, q0, 8, 1.0, 1e-13, 1e-12, 20, 5000, "direct")
    assert r.status == F.STATUS_OK
    assert r.m_found == len(ref_vals) == 7
    assert M.eig_relerr(r.evals, ref_vals) < 1e-12
    assert M.sin_theta(r.evecs, ref_vecs) < 1e-9
    assert M.orth_err(r.q_all) < 1e-12
    assert np.all(r.resid <= 1e-12)


@pytest.mark.parametrize("form", ["direct", "correction"])
def test_feast_random_spd_dense(form):
    a = _random_spd(250, 3)
    lam, v = np.linalg.eigh(a.toarray())
    lmin, lmax = 0.5 * (lam[4] + lam[5]), 0.5 * (lam[14] + lam[15])
    q0 = F.random_start(250, 16, 2)
    r = F.feast(a, lmin, lmax, q0, 4, 1.0, 1e-12, 1e-11, 40, 5000, form)
    assert r.status == F.STATUS_OK and r.m_found == 10
    assert M.eig_relerr(r.evals, lam[5:15]) < 1e-11
    assert M.sin_theta(r.evecs, v[:, 5:15]) < 1e-8


def test_courant_fischer():
    a = _random_spd(120, 4)
    lam = np.linalg.eigvalsh(a.toarray())
    for seed in range(3):
        q = F.random_start(120, 9, seed)
        ritz, _, _ = F.rayleigh_ritz(a, q)
        assert np.all(ritz >= lam[:9] - 1e-12)
        assert np.all(ritz <= lam[-9:] + 1e-12)


@pytest.mark.parametrize("m0,nc", [(5, 2), (6, 1), (5, 1)])
def test_outer_contraction_rate(m0, nc):
    n, cnt = 80, 5
    a = G.path(n).scipy()
    lam = E.path_eigenvalues(n)
    lmin, lmax = -0.01, 0.5 * (lam[cnt - 1] + lam[cnt])
    z, w = Q.nodes(lmin, lmax, nc, 1.0)
    f = np.abs(Q.filter_value(lam, z, w))
    rate = np.sort(f)[::-1][m0] / f[:cnt].min()
    vecs = np.stack([E.path_eigenvector(n, k) for k in range(cnt)], axis=1)
    q = F.random_start(n, m0, 5)
    errs = []
    for _ in range(10):
        r = F.feast(a, lmin, lmax, q, nc, 1.0, 1e-14, 0.0, 1, 5000, "direct")
        q = r.q_all
        errs.append(M.sin_theta(r.q_all[:, :cnt], vecs))
    ratios = np.array(errs[6:]) / np.array(errs[5:-1])
    assert 0.1 < rate < 0.9
    assert np.all(np.abs(ratios / rate - 1.0) < 0.1)


def test_warmstart_map_properties():
    a = G.grid2d(6, 7, 0.01).scipy()
    glo, ghi = F.gershgorin(a)
    s, t, name = F.warmstart_map(a, 0.02, 0.5, "low")
    assert name == "low"
    assert abs(s * 0.02 + t - 1.0) < 1e-14 and abs(s * ghi + t) < 1e-14
    s, t, name = F.warmstart_map(a, 0.02, 0.5, "literal")
    assert abs(s * 0.02 + t) < 1e-14 and abs(s * 0.5 + t - 1.0) < 1e-14
    assert F.warmstart_map(a, 0.02, 0.5, "auto")[2] == "low"
    assert F.warmstart_map(a, ghi - 1.0, ghi, "auto")[2] == "literal"
    lam = np.linalg.eigvalsh(a.toarray())
    assert glo <= lam.min() + 1e-12 and ghi >= lam.max() - 1e-12


def test_warmstart_halko_davis_kahan_bound():
    # A with spectrum in [lmin, lmax], target = top m0 (Assumption 1.2-1.3)
    n, m0, p, q = 300, 6, 10, 1
    rng = np.random.default_rng(9)
    v, _ = np.linalg.qr(rng.standard_normal((n, n)))
    beta = np.concatenate([np.linspace(1.0, 0.9, m0), np.linspace(0.45, 0.0, n - m0)])
    lmin, lmax = 2.0, 5.0
    lam = lmin + beta * (lmax - lmin)
    a = sp.csr_matrix((v * lam) @ v.T)
    om = P.gaussian_matrix(n, m0 + p, 4)
    s, t, _ = F.warmstart_map(a, lmin, lmax, "literal")
    y = s * (a @ om) + t * om
    for _ in range(q):
        y = s * (a @ (s * (a @ y) + t * y)) + t * (s * (a @ y) + t * y)
    qy = F.orthonormalize(y)
    target = v[:, np.argsort(lam)[::-1][:m0]]
    err = np.linalg.norm(target - qy @ (qy.T @ target), 2)
    delta = 1e-3
    c1 = 1.0 + 0.5 * p * np.log(2 * m0 / delta)
    bm, bm1 = 0.9, 0.45
    r_halko = c1 * np.sqrt(1 + m0 / (p - 1)) * bm1 * (bm1 / bm) ** (2 * q)
    assert err <= r_halko / (bm - bm1)
    q0, theta, info = F.warmstart(a, lmin, lmax, m0, p, q, om, "literal")
    assert q0.shape == (n, m0) and M.orth_err(q0) < 1e-12
    # truncation keeps the m0 Ritz values closest to the interval centre
    ritz = info["ritz_all"]
    c = 0.5 * (lmin + lmax)
    far = np.sort(np.abs(ritz - c))[m0 - 1]
    assert np.all(np.abs(theta - c) <= far + 1e-15)
    assert np.allclose(np.sort(theta), np.sort(ritz[np.argsort(np.abs(ritz - c))[:m0]]))


def test_warmstart_powers_help_low_end():
    a = G.grid2d(20, 20, 0.01).scipy()
    vals, _ = E.grid_spectrum((20, 20), 0.01)
    lmin, lmax = 0.005, 0.5 * (vals[5] + vals[6])
    _, vecs = E.grid_eigvecs_in((20, 20), 0.01, lmin, lmax)
    om = P.gaussian_matrix(400, 16, 0)
    errs = []
    for q in [0, 4, 40]:
        q0, _, _ = F.warmstart(a, lmin, lmax, 6, 10, q, om, "low")
        errs.append(np.linalg.norm(vecs - q0 @ (q0.T @ vecs), 2))
    assert errs[2] < errs[1] < errs[0]


def test_status_codes():
    a = G.path(60).scipy()
    lam = E.path_eigenvalues(60)
    q0 = F.random_start(60, 6, 0)
    # empty interval
    lo, hi = 0.5 * (lam[10] + lam[11]) + 1e-9, 0.5 * (lam[10] + lam[11]) + 2e-9
    r = F.feast(a, lo, hi, q0, 4, 1.0, 1e-12, 1e-10, 3, 2000)
    assert r.status == F.STATUS_NO_EIGENVALUE and r.m_found == 0
    # more eigenvalues inside than m0
    r = F.feast(a, -0.1, 0.5 * (lam[9] + lam[10]), q0, 8, 1.0, 1e-12, 1e-10, 8, 2000)
    assert r.status == F.STATUS_M0_TOO_SMALL
    # iteration cap
    r = F.feast(a, -0.1, 0.5 * (lam[2] + lam[3]), q0, 2, 1.0, 1e-12, 1e-15, 1, 2000)
    assert r.status == F.STATUS_NO_CONVERGENCE and r.outer_iters == 1


@pytest.mark.slow
def test_rafeast_correction_reaches_tight_tol_with_relaxed_solves():
    # relaxed inner tolerance 1e-4, tight outer tolerance (Section 3.1 Phase 2)
    lap = G.knn3d(1500, 8, seed=3, shift=1e-3)
    a = lap.scipy()
    lam, v = np.linalg.eigh(a.toarray())
    k = 12
    lmin, lmax = 0.5 * lam[0], 0.5 * (lam[k - 1] + lam[k])
    r = F.rafeast(a, lmin, lmax, 18, 10, 2, 1, 2, 1.0, 1e-4, 1e-11, 40, 5000,
                  "correction")
    assert r.status == F.STATUS_OK and r.m_found == k
    assert M.eig_relerr(r.evals, lam[:k]) < 1e-11
    assert M.sin_theta(r.evecs, v[:, :k]) < 1e-8


def test_one_norm_hand_computed():
    """||A||_1 is the largest column sum of absolute values (the convergence
    test's normalisation, Algorithm 1's "until convergence" as read here).
    The matrices separate it from the row-sum, Frobenius and spectral norms
    and from a sum without absolute values."""
    # path Laplacian P5: column sums of |a_ij| are 2, 4, 4, 4, 2
    a = G.path(5).scipy()
    assert F.one_norm(a) == 4.0
    # ||A||_2 = 2 - 2 cos(4 pi / 5) = 3.618..., ||A||_F = sqrt(22)
    assert abs(np.linalg.norm(a.toarray(), 2) - (2 - 2 * np.cos(4 * np.pi / 5))) < 1e-12
    # a diagonal shift adds to every column sum
    assert F.one_norm(G.path(5, shift=0.5).scipy()) == 4.5
    # columns (1, 7), rows (6, 2): the 1-norm is 7, the infinity-norm 6
    assert F.one_norm(sp.csr_matrix(np.array([[1.0, 5.0], [0.0, 2.0]]))) == 7.0
    # negative entries count by their size: |.| column sums (5, 2), plain (-1, 0)
    assert F.one_norm(sp.csr_matrix(np.array([[-3.0, 1.0], [2.0, -1.0]]))) == 5.0


def test_residuals_hand_computed():
    """res_i = ||A q_i - lam_i q_i||_2 / ||A||_1, worked by hand on the path
    Laplacian P5 (||A||_1 = 4):
    * q = e_0, lam = 1: A e_0 - e_0 = (0, -1, 0, 0, 0), res = 1/4;
    * q = e_2, lam = 2: A e_2 - 2 e_2 = (0, -1, 0, -1, 0), res = sqrt(2)/4
      (a max-norm would give 1/4, a 1-norm 2/4);
    * q = e_2, lam = 0: (0, -1, 2, -1, 0), res = sqrt(6)/4;
    * q = (1,...,1)/sqrt(5), lam = 0.5: A q = 0, res = 0.5/4.
    With a shift of 0.5 every column sum grows by 0.5 and A e_0 = 1.5 e_0 - e_1."""
    a = G.path(5).scipy()
    e = np.eye(5)
    q = np.stack([e[0], e[2], e[2], np.ones(5) / np.sqrt(5)], axis=1)
    lam = np.array([1.0, 2.0, 0.0, 0.5])
    expect = np.array([1.0, np.sqrt(2.0), np.sqrt(6.0), 0.5]) / 4.0
    assert np.allclose(F.residuals(a, lam, q), expect, rtol=0, atol=1e-15)
    # the same with A Q and ||A||_1 passed in
    assert np.allclose(F.residuals(a, lam, q, aq=a @ q, norm_a=4.0), expect, rtol=0, atol=1e-15)
    s = G.path(5, shift=0.5).scipy()
    got = F.residuals(s, np.array([1.5, 0.0]), np.stack([e[0], e[0]], axis=1))
    assert np.allclose(got, np.array([1.0, np.sqrt(1.5 ** 2 + 1.0)]) / 4.5, rtol=0, atol=1e-15)
