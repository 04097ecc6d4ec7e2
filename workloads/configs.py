"""The five benchmark workloads (seeded synthetic inputs, no method arithmetic).

Each config names the matrix generator, the solver parameters and where its
search interval comes from. Intervals that need a spectrum pre-pass are read
from ``tests/golden/spectra.json`` (written by ``tests/golden/make_golden.py``
with the oracle's exact eigensolvers); the closed-form ones are stored there
too, so every consumer reads the same numbers.

* ``grid2d``  plain FEAST, FP64: 2-D 5-point grid 40x50 (n=2000, nnz=9820),
  16 smallest nonzero eigenvalues, m0=24, N_c=8, COCG tol 1e-10, outer 1e-10,
  random start from seed 0.
* ``knn8k``   RA-FEAST, FP64: kNN graph, 8000 uniform points in [0,1]^3
  (seed 1), k=10, union-symmetrised, unit weights, + 1e-3 I; the 32 smallest
  eigenvalues; p=10, q=2, m0=42, N_c=2, COCG tol 1e-4, outer 1e-10. Compared
  with plain FEAST at N_c=8, COCG tol 1e-10 on the same matrix.
* ``knn200k`` RA-FEAST, mixed: the same construction with n=200,000 (seed 2),
  64 smallest eigenvalues, m0=80, N_c=4, p=20, q=2, relaxed inner solves
  (COCG tolerance 1e-2, at most 100 steps), outer tolerance 1e-11.
* ``grid3d``  RA-FEAST, mixed: 3-D 7-point grid 100^3 (n=1e6, nnz=6.94e6)
  + 1e-2 I, 63 eigenvalues in [0.005, 0.0272568], m0=96, N_c=4, p=20, q=2,
  inner solves as ``knn200k``, outer tolerance 1e-10.
* ``rgg2k``, ``rgg8k``, ``rgg16k``: the paper's own workload (Section 5.1),
  random geometric graphs in the unit square with r = 1.5 sqrt(log n / n),
  L = D - A, the eigenvalues in [0.001, 5.0] (12, 29, 46 of them), subspace
  1.5 x count, RA-FEAST FP64 at N_c = 2, p=10, q=2, COCG tolerance 1e-4,
  max_iter = 4.
* ``sbm64``   batched RA-FEAST, mixed: 64 stochastic-block-model Laplacians
  + 1e-3 I, n log-uniform in [2000, 300000] (seed 4), 4..16 blocks,
  p_in = 20/n_block, p_out = 1/n, k = blocks + 8, m0 = ceil(1.5 k), N_c=2;
  half-ellipse ratio e = 0.3, inner solves as ``knn200k``, outer tolerance
  1e-10 (SBM_SOLVE), warmstart p=10, q=2 with each instance's own seed.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os

import numpy as np

from . import graphs

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "tests", "golden", "spectra.json")


@dataclasses.dataclass
class Config:
    key: str
    make: callable          # () -> graphs.Laplacian
    count: int              # eigenvalues inside the interval
    m0: int
    nc: int
    precision: str          # "fp64" | "mixed"
    solve_tol: float
    outer_tol: float
    form: str               # "direct" | "correction"
    warmstart: bool
    p: int = 0
    q: int = 0
    seed: int = 0
    e: float = 1.0
    max_outer: int = 40
    max_inner: int = 20000
    description: str = ""


def _cfgs():
    return {
        "grid2d": Config("grid2d", lambda: graphs.grid2d(40, 50, 0.0), 16, 24, 8,
                         "fp64", 1e-10, 1e-10, "direct", False, seed=0,
                         description="plain FEAST FP64, 2-D grid 40x50"),
        "knn8k": Config("knn8k", lambda: graphs.knn3d(8000, 10, 1, 1e-3), 32, 42, 2,
                        "fp64", 1e-4, 1e-10, "correction", True, p=10, q=2, seed=1,
                        description="RA-FEAST FP64, kNN n=8000"),
        "knn8k_plain": Config("knn8k_plain", lambda: graphs.knn3d(8000, 10, 1, 1e-3),
                              32, 42, 8, "fp64", 1e-10, 1e-10, "direct", False,
                              seed=1, description="plain FEAST FP64 N_c=8, kNN n=8000"),
        # the float32 inner solves are capped at 60 COCG steps: a sweep of caps
        # 40..130 on the GPU path gave the shortest solves there (fewer steps
        # per outer iteration outweigh the three extra outer iterations), with
        # the same eigenvalue errors
        "knn200k": Config("knn200k", lambda: graphs.knn3d(200000, 10, 2, 1e-3), 64, 80, 4,
                          "mixed", 1e-2, 1e-11, "correction", True, p=20, q=2, seed=2,
                          max_inner=60, description="RA-FEAST mixed, kNN n=200000"),
        # outer tolerance 1e-10: the measured residual sequence is 2.9e-10,
        # 1.02e-11, 1.1e-12 at outer iterations 8, 9, 10, so 1e-11 would put the
        # stopping step on the fourth digit of a residual; the eigenvalues are
        # at 3e-14 relative error by then. The inner cap stays at 100: at 60 the
        # solve is 17% shorter but stops on a residual just under 1e-10, where
        # the Davis-Kahan bound on the eigenspace (1.1e-6) no longer shows the
        # 1e-6 gate (at 100: 1.7e-7)
        "grid3d": Config("grid3d", lambda: graphs.grid3d(100, 100, 100, 1e-2), 63, 96, 4,
                         "mixed", 1e-2, 1e-10, "correction", True, p=20, q=2, seed=3,
                         max_inner=100, description="RA-FEAST mixed, 3-D grid 100^3"),
        # the paper's experiment (Section 5.1): random geometric graph in the
        # unit square, r = 1.5 sqrt(log n / n), L = D - A (no shift), the
        # eigenvalues in [0.001, 5.0]; subspace 1.5 x their count (46 at
        # n = 16,000); RA-FEAST FP64 with relaxed solves and the paper's
        # iteration limit max_iter = 4 (bench.py adds the other N_c / max_iter
        # rows of Table 1 and standard FEAST)
        "rgg16k": Config("rgg16k", lambda: graphs.rgg2d(16000, seed=0), 46, 69, 2, "fp64",
                         1e-4, 1e-10, "correction", True, p=10, q=2, seed=1, max_outer=4,
                         max_inner=2000, description="RA-FEAST FP64, RGG n=16000 (Section 5.1)"),
        "rgg2k": Config("rgg2k", lambda: graphs.rgg2d(2000, seed=0), 12, 18, 2, "fp64",
                        1e-4, 1e-10, "correction", True, p=10, q=2, seed=1, max_outer=4,
                        max_inner=2000, description="RA-FEAST FP64, RGG n=2000 (Section 5.1)"),
        "rgg8k": Config("rgg8k", lambda: graphs.rgg2d(8000, seed=0), 29, 44, 2, "fp64",
                        1e-4, 1e-10, "correction", True, p=10, q=2, seed=1, max_outer=4,
                        max_inner=2000, description="RA-FEAST FP64, RGG n=8000 (Section 5.1)"),
    }


CONFIGS = _cfgs()


# solver settings of every instance of the batched SBM sweep. The intervals
# end inside the dense low edge of these spectra, so at N_c = 2 the filter's
# contraction is poor on a circle (e = 1: 0.65-0.89 per outer iteration on
# sampled instances; the oracle needs 186 iterations on instance 8). The
# flatter ellipse of FEAST's Hermitian default (ratio 0.3) brings it to
# 0.38-0.72 (67 iterations on instance 8). A 1e-10 residual bounds the
# eigenvalue error far below the 1e-8 gate (the error enters squared).
SBM_SOLVE = dict(nc=2, e=0.3, precision="mixed", solve_tol=1e-2, outer_tol=1e-10,
                 form="correction", p=10, q=2, max_outer=150, max_inner=100)


def sbm_instances(count: int = 64, seed: int = 4, n_lo: int = 2000,
                  n_hi: int = 300000):
    """Parameters of the batched SBM sweep: list of dicts with n, blocks,
    block sizes, p_in, p_out, k, m0 and a per-instance seed."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kb = int(rng.integers(4, 17))
        base = n // kb
        sizes = [base + (1 if b < n - base * kb else 0) for b in range(kb)]
        nb = n / kb
        k = kb + 8
        out.append(dict(index=t, n=n, blocks=kb, sizes=sizes, p_in=20.0 / nb,
                        p_out=1.0 / n, k=k, m0=int(math.ceil(1.5 * k)),
                        seed=seed * 1000 + t))
    return out


def make_sbm(inst) -> graphs.Laplacian:
    return graphs.sbm(inst["sizes"], inst["p_in"], inst["p_out"], inst["seed"], 1e-3)


def load_golden():
    if not os.path.exists(GOLDEN):
        raise FileNotFoundError(f"missing {GOLDEN}; run tests/golden/make_golden.py")
    with open(GOLDEN) as f:
        return json.load(f)


def interval(key: str):
    """(lmin, lmax) of a config from the stored spectrum pre-pass."""
    g = load_golden()[key]
    return g["lmin"], g["lmax"]
