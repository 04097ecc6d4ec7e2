"""The C-ABI library builds, loads and exports every function the header
declares (CPU only: no compute call is made without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rafeast.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(rafeast_\w+)\s*\(", text,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2512_01257_gb300 import build, rafeast
    if not os.path.exists(rafeast.LIB_PATH):
        build.build()
    return rafeast.LIB_PATH


def test_header_declares_the_hot_path():
    names = _declared()
    for must in ["rafeast_create", "rafeast_warmstart", "rafeast_solve", "rafeast_destroy",
                 "rafeast_status_string", "rafeast_solve_batched", "rafeast_filter",
                 "rafeast_spmm", "rafeast_orthonormalize", "rafeast_rayleigh_ritz"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rafeast_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_maps_statuses(libpath):
    from paper_2512_01257_gb300 import rafeast as R
    lib = R.load()
    for name in _declared():
        assert hasattr(lib, name)
    assert R.status_string(0) == "ok"
    assert "breakdown" in R.status_string(R.RAFEAST_ERR_COCG_BREAKDOWN)
    assert R.status_string(12345) == "unknown status"


def test_quadrature_entry_matches_oracle_on_host(libpath):
    # rafeast_quadrature is pure host code: safe to call without a GPU
    import numpy as np
    from oracle import quadrature as Q
    from paper_2512_01257_gb300 import rafeast as R
    for nc in [1, 2, 3, 4, 8, 16, 40]:
        for e in [1.0, 0.3]:
            z, w = R.rafeast_quadrature(0.01, 0.8, nc, e)
            z2, w2 = Q.nodes(0.01, 0.8, nc, e)
            assert np.allclose(z, z2, rtol=0, atol=1e-15)
            assert np.allclose(w, w2, rtol=0, atol=1e-15)
    with pytest.raises(R.RafeastError):
        R.rafeast_quadrature(1.0, 0.5, 4)
