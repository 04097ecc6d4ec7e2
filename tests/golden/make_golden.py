"""Write tests/golden/spectra.json: intervals and reference eigenvalues.

Calls only the oracle (``oracle.exact``) and the seeded generators. For each
workload it records the matrix checksum, the search interval (gap midpoints
of the exact spectrum: below the smallest eigenvalue, lmin = half of it; the
upper end midway between the k-th and (k+1)-th eigenvalues), the number of
eigenvalues inside, and the reference eigenvalues (inside plus a few on each
side). Sources: closed form for the grids, ARPACK shift-invert for the kNN
graphs, Lanczos (ARPACK, smallest algebraic) for the SBM instances.

    python tests/golden/make_golden.py [keys...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exact as E  # noqa: E402
from workloads import configs as C  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spectra.json")


def _entry(lap, vals, k, source, lmin=None, lmax=None, extra=4):
    vals = np.sort(np.asarray(vals))
    if lmin is None:
        lmin = 0.5 * vals[0]
    if lmax is None:
        lmax = 0.5 * (vals[k - 1] + vals[k])
    inside = vals[(vals >= lmin) & (vals <= lmax)]
    return dict(n=lap.n, nnz=lap.nnz, checksum=lap.checksum(), lmin=float(lmin),
                lmax=float(lmax), count=int(inside.size),
                evals=[float(v) for v in inside],
                neighbours=[float(v) for v in vals[(vals > lmax)][:extra]],
                gap_right=float(vals[vals > lmax][0] - inside.max()),
                source=source)


def grid2d():
    cfg = C.CONFIGS["grid2d"]
    lap = cfg.make()
    vals, _ = E.grid_spectrum((40, 50), 0.0)
    return _entry(lap, vals[:64], 16, "closed form 4-2cos(pi a/40)-2cos(pi b/50)",
                  lmin=0.0019733, lmax=0.0792439)


def grid3d():
    cfg = C.CONFIGS["grid3d"]
    lap = cfg.make()
    vals, _ = E.grid_spectrum((100, 100, 100), 0.01)
    return _entry(lap, vals[:200], 63, "closed form 0.01+sum of three 2-2cos(pi k/100)",
                  lmin=0.005, lmax=0.5 * (0.0267692 + 0.0277444))


def knn(key, k, nev):
    lap = C.CONFIGS[key].make()
    t = time.time()
    vals, vecs = E.eigsh_smallest(lap.scipy(), nev, sigma=0.0, tol=1e-14)
    res = np.linalg.norm(lap.scipy() @ vecs - vecs * vals, axis=0).max()
    ent = _entry(lap, vals, k, "ARPACK shift-invert (SuperLU, MMD order)")
    ent["max_residual"] = float(res)
    ent["seconds"] = time.time() - t
    return ent


def rgg(key):
    """The paper's interval [0.001, 5.0] on an RGG Laplacian (ARPACK
    shift-invert just below the zero eigenvalue)."""
    lap = C.CONFIGS[key].make()
    t = time.time()
    vals, vecs = E.eigsh_smallest(lap.scipy(), C.CONFIGS[key].m0 + 6, sigma=-0.01, tol=1e-14)
    res = np.linalg.norm(lap.scipy() @ vecs - vecs * vals, axis=0).max()
    ent = _entry(lap, vals, 0, "ARPACK shift-invert (SuperLU, MMD order)", lmin=0.001, lmax=5.0)
    ent["max_residual"] = float(res)
    ent["seconds"] = time.time() - t
    return ent


def sbm64():
    """The 64 stochastic-block-model instances of the batched sweep: per
    instance the k = blocks + 8 smallest eigenvalues, the interval's upper end
    midway to eigenvalue k+1 (moved up while that gap is below 1e-6 of
    lambda_k), lmin half the smallest eigenvalue."""
    out = []
    for inst in C.sbm_instances():
        lap = C.make_sbm(inst)
        a = lap.scipy()
        t = time.time()
        k = inst["k"]
        vals, vecs = E.eigsh_smallest_lanczos(a, k + 6, tol=1e-13, seed=inst["seed"])
        while vals[k] - vals[k - 1] < 1e-6 * vals[k - 1] and k + 1 < vals.size:
            k += 1
        res = np.linalg.norm(a @ vecs - vecs * vals, axis=0).max()
        ent = _entry(lap, vals, k, "ARPACK Lanczos, smallest algebraic", extra=5)
        ent.update(index=inst["index"], blocks=inst["blocks"], k=k, m0=inst["m0"],
                   max_residual=float(res), seconds=time.time() - t)
        print(" sbm", inst["index"], lap.n, ent["count"], "%.1fs" % ent["seconds"], flush=True)
        out.append(ent)
    return dict(instances=out, source="ARPACK Lanczos, smallest algebraic")


def main(keys):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    makers = {
        "grid2d": grid2d,
        "grid3d": grid3d,
        "knn8k": lambda: knn("knn8k", 32, 44),
        "knn200k": lambda: knn("knn200k", 64, 76),
        "sbm64": sbm64,
        "rgg2k": lambda: rgg("rgg2k"),
        "rgg8k": lambda: rgg("rgg8k"),
        "rgg16k": lambda: rgg("rgg16k"),
    }
    for key in keys or list(makers):
        print("computing", key, flush=True)
        data[key] = makers[key]()
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)
        if "count" in data[key]:
            print(key, data[key]["count"], data[key]["lmin"], data[key]["lmax"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
