"""rafeast_solve_batched: stochastic-block-model problems of uneven n solved
together (grouped COCG launches), checked against the definition (ARPACK
Lanczos from the oracle) and against rafeast_solve one problem at a time."""
import numpy as np
import pytest

from oracle import exact as E
from oracle import metrics as M
from workloads import configs as CF

pytestmark = pytest.mark.gpu


def _problems(count, seed, n_lo, n_hi):
    """Seeded SBM instances with their intervals (gap midpoints of the
    Lanczos spectrum) and reference eigenpairs."""
    out = []
    for inst in CF.sbm_instances(count=count, seed=seed, n_lo=n_lo, n_hi=n_hi):
        lap = CF.make_sbm(inst)
        k = inst["k"]
        w, v = E.eigsh_smallest_lanczos(lap.scipy(), k + 4, seed=inst["seed"])
        assert w[k] - w[k - 1] > 1e-6 * w[k - 1]
        lmin, lmax = 0.5 * w[0], 0.5 * (w[k - 1] + w[k])
        out.append(dict(inst=inst, lap=lap, k=k, lmin=lmin, lmax=lmax, evals=w[:k],
                        evecs=v[:, :k]))
    return out


@pytest.fixture(scope="module")
def sbm6():
    return _problems(6, 21, 600, 6000)


def _handles(lib, probs, warm=True):
    hs = []
    S = CF.SBM_SOLVE
    for pr in probs:
        lap = pr["lap"]
        h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
        if warm:
            lib.rafeast_warmstart(h, pr["lmin"], pr["lmax"], pr["inst"]["m0"], S["p"], S["q"],
                                  pr["inst"]["seed"])
        hs.append(h)
    return hs


def _params(lib, pr, prec, **kw):
    S = dict(CF.SBM_SOLVE)
    S.update(kw)
    p = lib.RAFEAST_FP64 if prec == "fp64" else lib.RAFEAST_MIXED
    return lib.make_params(pr["lmin"], pr["lmax"], pr["inst"]["m0"], S["nc"], S["e"],
                           S["solve_tol"], S["outer_tol"], S["max_outer"], S["max_inner"], p,
                           lib.RAFEAST_FORM_CORRECTION, lib.RAFEAST_START_SUBSPACE)


def _run_batched(lib, hs, probs, prms):
    ev = [np.zeros(pr["inst"]["m0"]) for pr in probs]
    vec = [np.zeros((pr["inst"]["m0"], pr["lap"].n)) for pr in probs]
    res = [np.zeros(pr["inst"]["m0"]) for pr in probs]
    st, mf, info = lib.rafeast_solve_batched(hs, prms, ev, vec, res)
    return st, mf, info, ev, vec, res


@pytest.mark.parametrize("update", [1, 2])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batched_sbm_against_lanczos(lib, sbm6, prec, update):
    """update 1: grouped gathering update; 2: grouped streamed update (the
    first handle's option decides for the batch)."""
    hs = _handles(lib, sbm6)
    lib.rafeast_set_option(hs[0], lib.RAFEAST_OPT_UPDATE, update)
    try:
        prms = [_params(lib, pr, prec, solve_tol=1e-2 if prec == "mixed" else 1e-4,
                        max_inner=100 if prec == "mixed" else 2000) for pr in sbm6]
        st, mf, info, ev, vec, res = _run_batched(lib, hs, sbm6, prms)
        tol_e, tol_v = (1e-10, 1e-8) if prec == "fp64" else (1e-8, 1e-6)
        for t, pr in enumerate(sbm6):
            assert st[t] == lib.RAFEAST_OK, (t, info[t].as_dict())
            assert mf[t] == pr["k"]
            assert M.eig_relerr(ev[t][:mf[t]], pr["evals"]) <= tol_e
            assert M.sin_theta(vec[t][:mf[t]].T, pr["evecs"]) <= tol_v
            assert np.all(res[t][:mf[t]] <= CF.SBM_SOLVE["outer_tol"])
        # the grouped launches are counted once, in the first problem's info
        assert info[0].spmm_launches > max(i.spmm_launches for i in info[1:])
    finally:
        for h in hs:
            lib.rafeast_destroy(h)


def test_batched_equals_one_at_a_time(lib, sbm6):
    hs = _handles(lib, sbm6)
    hs1 = _handles(lib, sbm6)
    try:
        prms = [_params(lib, pr, "fp64", solve_tol=1e-4, max_inner=2000) for pr in sbm6]
        st, mf, info, ev, vec, res = _run_batched(lib, hs, sbm6, prms)
        for t, pr in enumerate(sbm6):
            m0 = pr["inst"]["m0"]
            e1, v1, r1 = np.zeros(m0), np.zeros((m0, pr["lap"].n)), np.zeros(m0)
            s1, mf1, inf1 = lib.rafeast_solve(hs1[t], prms[t], e1, v1, r1)
            assert s1 == st[t] == lib.RAFEAST_OK
            assert mf1 == mf[t]
            # same method and starting subspace; only reduction orders differ
            assert abs(inf1.outer_iters - info[t].outer_iters) <= 1
            assert M.eig_relerr(ev[t][:mf[t]], e1[:mf1]) <= 1e-10
            assert M.sin_theta(vec[t][:mf[t]].T, v1[:mf1].T) <= 1e-8
    finally:
        for h in hs + hs1:
            lib.rafeast_destroy(h)


def test_batched_per_problem_status(lib, sbm6):
    probs = sbm6[:3]
    hs = _handles(lib, probs)
    try:
        # the middle problem cannot meet outer_tol = 0: it stops at its own
        # max_outer with status 2 while the others converge
        prms = [_params(lib, pr, "mixed") for pr in probs]
        prms[1] = _params(lib, probs[1], "mixed", outer_tol=0.0, max_outer=2)
        st, mf, info, ev, vec, res = _run_batched(lib, hs, probs, prms)
        assert st[0] == st[2] == lib.RAFEAST_OK
        assert st[1] == lib.RAFEAST_NO_CONVERGENCE and info[1].outer_iters == 2
        assert M.eig_relerr(ev[0][:mf[0]], probs[0]["evals"]) <= 1e-8
    finally:
        for h in hs:
            lib.rafeast_destroy(h)


def test_batched_argument_errors(lib, sbm6):
    probs = sbm6[:2]
    hs = _handles(lib, probs)
    try:
        prms = [_params(lib, probs[0], "mixed"), _params(lib, probs[1], "fp64")]
        with pytest.raises(lib.RafeastError) as ei:
            _run_batched(lib, hs, probs, prms)
        assert ei.value.code == lib.RAFEAST_ERR_INVALID_ARG
        prms = [_params(lib, probs[0], "mixed"), _params(lib, probs[0], "mixed")]
        with pytest.raises(lib.RafeastError) as ei:
            _run_batched(lib, [hs[0], hs[0]], [probs[0], probs[0]], prms)
        assert ei.value.code == lib.RAFEAST_ERR_INVALID_ARG
        assert lib.load().rafeast_solve_batched(0, None, None, None, None, None, None, 0, None,
                                                None) == 0
    finally:
        for h in hs:
            lib.rafeast_destroy(h)
