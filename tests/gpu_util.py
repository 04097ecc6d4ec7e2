"""Helpers shared by the GPU tests (no arithmetic of the method)."""
import numpy as np
import scipy.sparse as sp


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def colmajor_dev(x_nm):
    """numpy (n, m) -> CUDA tensor (m, n) = column-major n x m."""
    return to_dev(np.ascontiguousarray(np.asarray(x_nm, dtype=np.float64).T))


def from_colmajor(t):
    """CUDA/CPU tensor (m, n) -> numpy (n, m)."""
    return t.detach().cpu().numpy().T.copy()


def rand_sym_csr(n, seed, density=0.02, dense_row=True, empty_rows=3):
    """Random symmetric sparse matrix with empty rows and one dense row, as
    (row_ptr, col_idx, values) plus the scipy matrix."""
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="coo")
    m = (m + m.T).tocsr()
    m = m + sp.diags(rng.uniform(1.0, 2.0, n))
    m = m.tolil()
    if dense_row:
        r = n // 3
        vals = rng.standard_normal(n) * 0.01
        m[r, :] = vals
        m[:, r] = vals[:, None]
        m[r, r] = 5.0
    for e in range(empty_rows):
        r = (7 * e + 1) % n
        if r == n // 3:
            continue
        m[r, :] = 0
        m[:, r] = 0
    m = m.tocsr()
    m.eliminate_zeros()
    m.sort_indices()
    return (m.indptr.astype(np.int32), m.indices.astype(np.int32),
            m.data.astype(np.float64), m)


def set_solver(lib, h, solver):
    """0: one COCG per shift; 1: multi-shift COCG, update with gathered
    products; 2: multi-shift COCG, streamed update."""
    lib.rafeast_set_option(h, lib.RAFEAST_OPT_SOLVER, 0 if solver == 0 else 1)
    if solver:
        lib.rafeast_set_option(h, lib.RAFEAST_OPT_UPDATE, 1 if solver == 1 else 2)
