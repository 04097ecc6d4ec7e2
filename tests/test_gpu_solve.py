"""End-to-end parity of rafeast_solve with the definition (closed form /
ARPACK) and with the oracle, on the small workloads: plain FEAST FP64 on the
40x50 grid, RA-FEAST FP64 and mixed on the n=8000 kNN graph, status codes."""
import numpy as np
import pytest

from gpu_util import colmajor_dev, set_solver
from oracle import exact as E
from oracle import feast as OF
from oracle import metrics as M
from workloads import configs as CF
from workloads import graphs as G

pytestmark = pytest.mark.gpu


def _solve(lib, h, prm, n):
    m0 = prm.m0
    evals = np.zeros(m0)
    evecs = np.zeros((m0, n))
    resid = np.zeros(m0)
    st, mf, info = lib.rafeast_solve(h, prm, evals, evecs, resid)
    return st, mf, evals[:mf], evecs[:mf].T.copy(), resid[:mf], info


def test_grid2d_plain_feast_fp64(lib):
    cfg = CF.CONFIGS["grid2d"]
    lap = cfg.make()
    lmin, lmax = CF.interval("grid2d")
    ref_vals, ref_vecs = E.grid_eigvecs_in((40, 50), 0.0, lmin, lmax)
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
    try:
        prm = lib.make_params(lmin, lmax, cfg.m0, cfg.nc, 1.0, cfg.solve_tol, cfg.outer_tol,
                              cfg.max_outer, cfg.max_inner, lib.RAFEAST_FP64,
                              lib.RAFEAST_FORM_DIRECT, lib.RAFEAST_START_RANDOM, cfg.seed)
        st, mf, ev, vec, res, info = _solve(lib, h, prm, lap.n)
        assert st == lib.RAFEAST_OK, info.as_dict()
        assert mf == 16
        assert M.eig_relerr(ev, ref_vals) <= 1e-10
        assert M.sin_theta(vec, ref_vecs) <= 1e-8
        assert np.all(res <= cfg.outer_tol)
        # the oracle, same seeded start, same algorithm
        q0 = OF.random_start(lap.n, cfg.m0, cfg.seed)
        o = OF.feast(lap.scipy(), lmin, lmax, q0, cfg.nc, 1.0, cfg.solve_tol, cfg.outer_tol,
                     cfg.max_outer, cfg.max_inner, "direct")
        assert o.status == 0 and o.outer_iters == info.outer_iters
        assert M.eig_relerr(ev, o.evals) <= 1e-10
        assert M.sin_theta(vec, o.evecs) <= 1e-8
    finally:
        lib.rafeast_destroy(h)


@pytest.fixture(scope="module")
def knn8k():
    lap = CF.CONFIGS["knn8k"].make()
    g = CF.load_golden()["knn8k"]
    assert g["checksum"] == lap.checksum()
    w, v = E.eigsh_smallest(lap.scipy(), 32)
    assert np.allclose(w, g["evals"], rtol=1e-12)
    return lap, g, w, v


@pytest.mark.parametrize("solver", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_knn8k_rafeast(lib, knn8k, prec, solver):
    lap, g, w, v = knn8k
    cfg = CF.CONFIGS["knn8k"]
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
    set_solver(lib, h, solver)
    try:
        lib.rafeast_warmstart(h, g["lmin"], g["lmax"], cfg.m0, cfg.p, cfg.q, cfg.seed)
        p = lib.RAFEAST_FP64 if prec == "fp64" else lib.RAFEAST_MIXED
        prm = lib.make_params(g["lmin"], g["lmax"], cfg.m0, cfg.nc, 1.0, cfg.solve_tol,
                              cfg.outer_tol, cfg.max_outer, cfg.max_inner, p,
                              lib.RAFEAST_FORM_CORRECTION, lib.RAFEAST_START_SUBSPACE)
        st, mf, ev, vec, res, info = _solve(lib, h, prm, lap.n)
        assert st == lib.RAFEAST_OK, info.as_dict()
        assert mf == 32
        tol_e, tol_v = (1e-10, 1e-8) if prec == "fp64" else (1e-8, 1e-6)
        assert M.eig_relerr(ev, g["evals"]) <= tol_e
        assert M.sin_theta(vec, v) <= tol_v
    finally:
        lib.rafeast_destroy(h)


def test_knn8k_plain_nc8(lib, knn8k):
    lap, g, w, v = knn8k
    cfg = CF.CONFIGS["knn8k_plain"]
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
    try:
        prm = lib.make_params(g["lmin"], g["lmax"], cfg.m0, cfg.nc, 1.0, cfg.solve_tol,
                              cfg.outer_tol, cfg.max_outer, cfg.max_inner, lib.RAFEAST_FP64,
                              lib.RAFEAST_FORM_DIRECT, lib.RAFEAST_START_RANDOM, cfg.seed)
        st, mf, ev, vec, res, info = _solve(lib, h, prm, lap.n)
        assert st == lib.RAFEAST_OK, info.as_dict()
        assert mf == 32
        assert M.eig_relerr(ev, g["evals"]) <= 1e-10
        assert M.sin_theta(vec, v) <= 1e-8
    finally:
        lib.rafeast_destroy(h)


def test_status_codes(lib):
    lap = G.path(300)
    lam = E.path_eigenvalues(300)
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, 0.0)
    try:
        mid = 0.5 * (lam[40] + lam[41])
        prm = lib.make_params(mid + 1e-9, mid + 2e-9, 6, 4, 1.0, 1e-12, 1e-10, 3, 3000,
                              lib.RAFEAST_FP64, lib.RAFEAST_FORM_DIRECT)
        st, mf, *_ = _solve(lib, h, prm, lap.n)
        assert st == lib.RAFEAST_NO_EIGENVALUE and mf == 0
        prm = lib.make_params(-0.1, 0.5 * (lam[9] + lam[10]), 6, 8, 1.0, 1e-12, 1e-10, 6, 3000,
                              lib.RAFEAST_FP64, lib.RAFEAST_FORM_DIRECT)
        st, mf, *_ = _solve(lib, h, prm, lap.n)
        assert st == lib.RAFEAST_M0_TOO_SMALL and mf == 6
        # outer_tol = 0 cannot be met: stop at max_outer with the pairs found
        prm = lib.make_params(-0.1, 0.5 * (lam[2] + lam[3]), 6, 8, 1.0, 1e-12, 0.0, 2, 3000,
                              lib.RAFEAST_FP64, lib.RAFEAST_FORM_DIRECT)
        st, mf, ev, vec, res, info = _solve(lib, h, prm, lap.n)
        assert st == lib.RAFEAST_NO_CONVERGENCE and info.outer_iters == 2 and mf == 3
        # invalid arguments are rejected before any work
        bad = lib.make_params(1.0, 0.5, 6, 2)
        with pytest.raises(lib.RafeastError):
            _solve(lib, h, bad, lap.n)
        # N_c in 1..16 (one quadrature node per shifted solve)
        for nc in (0, 17):
            with pytest.raises(lib.RafeastError):
                _solve(lib, h, lib.make_params(0.0, 1.0, 6, nc), lap.n)
        # subspace start without a subspace of that size
        prm = lib.make_params(0.0, 0.1, 7, 2, start=lib.RAFEAST_START_SUBSPACE)
        with pytest.raises(lib.RafeastError):
            _solve(lib, h, prm, lap.n)
    finally:
        lib.rafeast_destroy(h)


def test_invalid_csr_rejected(lib):
    rp = np.array([0, 2, 3], dtype=np.int32)
    ci = np.array([0, 5, 1], dtype=np.int32)  # column 5 out of range
    va = np.ones(3)
    with pytest.raises(lib.RafeastError):
        lib.rafeast_create(rp, ci, va, 0.0)
    ci = np.array([0, 1, 0], dtype=np.int32)
    va = np.array([2.0, -1.0, -0.5])  # asymmetric values
    with pytest.raises(lib.RafeastError):
        lib.rafeast_create(rp, ci, va, 0.0, flags=lib.RAFEAST_CREATE_CHECK_SYMMETRY)
