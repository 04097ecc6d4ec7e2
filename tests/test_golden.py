"""The stored reference spectra (tests/golden/spectra.json, written by
tests/golden/make_golden.py with ARPACK or closed forms) checked against an
independent computation on the CPU: a dense symmetric eigendecomposition of
the regenerated matrix, for the stored workloads small enough for it. Also
the bookkeeping every GPU test relies on: the regenerated matrix is the one
the spectrum was computed for, the interval holds exactly the stored
eigenvalues, and its ends lie in gaps of the spectrum."""
import numpy as np
import pytest

from workloads import configs as CF


def _dense_spectrum(lap):
    return np.linalg.eigvalsh(lap.scipy().toarray())


def _check(g, w):
    lmin, lmax = g["lmin"], g["lmax"]
    inside = w[(w >= lmin) & (w <= lmax)]
    assert len(inside) == g["count"] == len(g["evals"])
    assert np.max(np.abs(inside - np.array(g["evals"]))) <= 1e-9 * max(1.0, abs(lmax))
    # the ends of the interval are not within 1e-6 of an eigenvalue
    assert np.min(np.abs(w - lmin)) > 1e-6 * max(abs(lmin), 1e-3)
    assert np.min(np.abs(w - lmax)) > 1e-6 * abs(lmax)
    if "neighbours" in g:
        above = w[w > lmax][: len(g["neighbours"])]
        assert np.max(np.abs(above - np.array(g["neighbours"]))) <= 1e-9 * max(1.0, abs(lmax))


@pytest.mark.parametrize("key", ["grid2d", "rgg2k"])
def test_small_stored_spectra_against_dense_eigh(key):
    cfg = CF.CONFIGS[key]
    g = CF.load_golden()[key]
    lap = cfg.make()
    assert lap.checksum() == g["checksum"]
    _check(g, _dense_spectrum(lap))


def test_smallest_sbm_instance_against_dense_eigh():
    gold = CF.load_golden()["sbm64"]["instances"]
    insts = CF.sbm_instances()
    t = int(np.argmin([i["n"] for i in insts]))
    assert insts[t]["n"] <= 4000
    lap = CF.make_sbm(insts[t])
    g = gold[t]
    assert lap.checksum() == g["checksum"]
    _check(g, _dense_spectrum(lap))
