"""Tiled seed dot kernel of the multi-shift COCG (float32, streamed update).

The tiled kernel stages each row tile's gathered rows in shared memory and
sums its dot products in a fixed order. These tests check it against the
oracle after a fixed number of COCG steps (Algorithm 2 Step 2a; no
convergence test, so a wrong alpha or beta cannot hide), against the
register-gather kernel on the same steps, for every column-block width, with
the shifted-direction updates of each step done by the update kernel or
deferred to the next dot kernel, on
unit Laplacians (values-free gathers) and on weighted matrices (values read),
with ragged column blocks, empty rows and a reordered kNN graph; and that two
solves with the same kernel shapes give identical results.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import colmajor_dev, from_colmajor, rand_sym_csr
from oracle import feast as OF
from oracle import quadrature as OQ
from workloads import graphs as G

pytestmark = pytest.mark.gpu

TILED_SHAPE = 1000000  # rafeast_profile's dots_shape of a tiled launch is above this


def _matrix(kind):
    """(row_ptr, col_idx, values, shift, scipy A incl. shift, interval)."""
    if kind == "grid":
        lap = G.grid2d(37, 41, shift=0.3)
        return lap.row_ptr, lap.col_idx, lap.values, lap.shift, lap.scipy(), (0.31, 0.6)
    if kind == "knn":
        lap = G.knn3d(3000, 10, 5, 1e-3)
        return lap.row_ptr, lap.col_idx, lap.values, lap.shift, lap.scipy(), (0.05, 0.4)
    if kind == "weighted":
        # a weighted Laplacian of the grid (values read by the kernel)
        lap = G.grid2d(29, 31, shift=0.2)
        a = lap.scipy(with_shift=False).tocsr()
        rng = np.random.default_rng(11)
        off = a.copy()
        off.setdiag(0)
        off.eliminate_zeros()
        off.data[:] = -rng.uniform(0.5, 1.5, off.nnz)
        off = (off + off.T) * 0.5
        wl = (sp.diags(-np.asarray(off.sum(axis=1)).ravel()) + off).tocsr()
        wl.sort_indices()
        return (wl.indptr.astype(np.int32), wl.indices.astype(np.int32), wl.data.copy(), 0.2,
                (wl + 0.2 * sp.identity(wl.shape[0])).tocsr(), (0.21, 0.5))
    # random symmetric matrix with empty rows (no diagonal entry either)
    rp, ci, va, a = rand_sym_csr(1531, 7, dense_row=False)
    d = a.diagonal()
    a = ((a - sp.diags(d)) * 0.02 + sp.diags(d)).tocsr()
    a.sort_indices()
    return (a.indptr.astype(np.int32), a.indices.astype(np.int32), a.data.copy(), 0.5,
            (a + 0.5 * sp.identity(a.shape[0])).tocsr(), (0.1, 0.4))


def _filter(lib, h, Q, m0, nc, lo, hi, steps, tiled, cb=0, defer=True):
    import torch
    # autotuning off: every step of the call runs the kernel asked for
    lib.rafeast_set_option(h, lib.RAFEAST_OPT_AUTOTUNE, 0)
    lib.rafeast_set_option(h, lib.RAFEAST_OPT_DEFER, 1 if defer else 0)
    lib.rafeast_set_option(h, lib.RAFEAST_OPT_SOLVER, 1)
    lib.rafeast_set_option(h, lib.RAFEAST_OPT_UPDATE, 2)
    lib.rafeast_set_option(h, lib.RAFEAST_OPT_TILED, 2 if tiled else 1)
    lib.rafeast_set_option(h, lib.RAFEAST_OPT_TILE_CB, cb)
    Qt = torch.zeros_like(Q)
    prm = lib.make_params(lo, hi, m0, nc, 1.0, 0.0, 1e-10, 1, steps, lib.RAFEAST_MIXED,
                          lib.RAFEAST_FORM_CORRECTION)
    info = lib.rafeast_filter(h, prm, Q, None, Qt)
    assert info.cocg_max_last == steps
    shape = lib.rafeast_profile(h, reset=False)["dots_shape"]
    assert (shape >= TILED_SHAPE) == tiled, shape
    if tiled and cb:
        assert (shape - TILED_SHAPE) // 100 == cb, shape
    return from_colmajor(Qt)


@pytest.mark.parametrize("kind", ["grid", "knn", "weighted", "empty_rows"])
@pytest.mark.parametrize("m0,nc", [(5, 2), (33, 4), (80, 4), (46, 3)])
def test_tiled_dots_match_oracle_and_gathers_stepwise(lib, kind, m0, nc):
    """12 fixed COCG steps: the tiled kernel (each block width) reproduces the
    oracle's filter as closely as the register-gather kernel does (both
    float32: within twice the gather kernel's error, floored at 5e-5), and
    the two float32 kernels agree with each other to float rounding."""
    rp, ci, va, shift, A, (lo, hi) = _matrix(kind)
    n = A.shape[0]
    h = lib.rafeast_create(rp, ci, va, shift)
    try:
        if kind == "knn":
            assert lib.rafeast_matrix_info(h)["order"] == 1  # bisection order chosen
        q0 = OF.random_start(n, m0, 1)
        Q = colmajor_dev(q0)
        z, w = OQ.nodes(lo, hi, nc, 1.0)
        exp, _ = OF.filter_apply(A, q0, z, w, 0.0, 12, "correction")
        scale = np.linalg.norm(exp)
        qg = _filter(lib, h, Q, m0, nc, lo, hi, 12, False)
        eg = np.linalg.norm(qg - exp) / scale
        tol = max(5e-5, 2.0 * eg)
        for cb in (4, 8):
            for defer in (True, False):
                qt = _filter(lib, h, Q, m0, nc, lo, hi, 12, True, cb, defer)
                et = np.linalg.norm(qt - exp) / scale
                assert et <= tol, (cb, defer, et, eg)
                assert np.linalg.norm(qt - qg) / scale <= max(2e-5, 2.0 * eg), (cb, defer)
    finally:
        lib.rafeast_destroy(h)


@pytest.mark.parametrize("kind", ["grid", "knn"])
def test_tiled_solves_are_reproducible(lib, kind):
    """The tiled kernel adds its dot products without atomics in a fixed
    order, so solves with the same kernel shapes give bit-identical
    eigenvalues, residuals and eigenvectors (autotuning off: one shape)."""
    import torch
    rp, ci, va, shift, A, _ = _matrix(kind)
    n = A.shape[0]
    lam = np.sort(np.linalg.eigvalsh(A.toarray()))
    # the interval ends in the widest relative gap after the 10th..14th value
    cnt = max(range(10, 15), key=lambda k: (lam[k] - lam[k - 1]) / lam[k])
    lmin, lmax = lam[0] * 0.5, 0.5 * (lam[cnt - 1] + lam[cnt])
    m0 = 24
    h = lib.rafeast_create(rp, ci, va, shift)
    try:
        lib.rafeast_set_option(h, lib.RAFEAST_OPT_AUTOTUNE, 0)
        lib.rafeast_set_option(h, lib.RAFEAST_OPT_TILED, 2)
        outs = []
        for _ in range(2):
            lib.rafeast_warmstart(h, lmin, lmax, m0, 10, 2, 3)
            prm = lib.make_params(lmin, lmax, m0, 4, 1.0, 1e-2, 1e-11, 40, 100,
                                  lib.RAFEAST_MIXED, lib.RAFEAST_FORM_CORRECTION,
                                  lib.RAFEAST_START_SUBSPACE)
            ev = np.zeros(m0)
            vec = np.zeros((m0, n))
            res = np.zeros(m0)
            st, mf, info = lib.rafeast_solve(h, prm, ev, vec, res)
            assert st == lib.RAFEAST_OK and mf == cnt
            assert lib.rafeast_profile(h, reset=False)["dots_shape"] >= TILED_SHAPE
            outs.append((ev.copy(), vec.copy(), res.copy(), info.outer_iters))
        (e1, v1, r1, i1), (e2, v2, r2, i2) = outs
        assert i1 == i2
        assert np.array_equal(e1, e2) and np.array_equal(r1, r2) and np.array_equal(v1, v2)
        assert np.max(np.abs(e1[:cnt] - lam[:cnt]) / lam[:cnt]) <= 1e-8
    finally:
        lib.rafeast_destroy(h)
