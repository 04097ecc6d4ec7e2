"""The paper's own workload (Section 5.1): random geometric graph Laplacians
in the unit square, the eigenvalues in [0.001, 5.0], against ARPACK
(tests/golden/spectra.json). RA-FEAST at the paper's contour sizes and
iteration limits reaches the accuracy the paper reports for them (maximum
absolute eigenvalue error below 1e-9); standard FEAST (random start, tight
solves) converges to the same eigenvalues."""
import numpy as np
import pytest

from workloads import configs as CF

pytestmark = pytest.mark.gpu


def _run(lib, key, nc, max_outer, warm=True, solve_tol=None):
    cfg = CF.CONFIGS[key]
    g = CF.load_golden()[key]
    lap = cfg.make()
    assert lap.checksum() == g["checksum"]
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
    try:
        if warm:
            lib.rafeast_warmstart(h, g["lmin"], g["lmax"], cfg.m0, cfg.p, cfg.q, cfg.seed)
        start = lib.RAFEAST_START_SUBSPACE if warm else lib.RAFEAST_START_RANDOM
        prm = lib.make_params(g["lmin"], g["lmax"], cfg.m0, nc, 1.0,
                              solve_tol or cfg.solve_tol, cfg.outer_tol, max_outer,
                              cfg.max_inner, lib.RAFEAST_FP64, lib.RAFEAST_FORM_CORRECTION, start,
                              cfg.seed)
        ev = np.zeros(cfg.m0)
        st, mf, info = lib.rafeast_solve(h, prm, ev, None, None)
        ref = np.array(g["evals"])
        assert mf == ref.size, (st, mf, info.as_dict())
        return st, float(np.max(np.abs(np.sort(ev[:mf]) - ref))), info
    finally:
        lib.rafeast_destroy(h)


@pytest.mark.parametrize("key", ["rgg2k", "rgg8k"])
@pytest.mark.parametrize("nc,max_outer", [(2, 4), (4, 4), (8, 2)])
def test_rgg_rafeast_paper_settings(lib, key, nc, max_outer):
    st, err, info = _run(lib, key, nc, max_outer)
    assert st in (lib.RAFEAST_OK, lib.RAFEAST_NO_CONVERGENCE)
    assert info.outer_iters <= max_outer
    assert err <= 1e-9, (err, info.as_dict())


def test_rgg_standard_feast(lib):
    st, err, info = _run(lib, "rgg2k", 8, 40, warm=False, solve_tol=1e-10)
    assert st == lib.RAFEAST_OK
    assert err <= 1e-10
