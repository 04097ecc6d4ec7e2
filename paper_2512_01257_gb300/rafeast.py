"""Python binding of librafeast (include/rafeast.h): argument marshalling only.

Every function has the name of the C entry point it calls. Device buffers are
torch CUDA tensors (PyTorch supplies memory and streams); host buffers are
numpy arrays. Dense blocks follow the C convention "column-major n x m":
they are passed as C-contiguous tensors/arrays of shape (m, n), row k holding
column k. The library must be built (``paper_2512_01257_gb300.build``);
loading fails loudly otherwise, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librafeast.so")

RAFEAST_OK = 0
RAFEAST_NO_EIGENVALUE = 1
RAFEAST_NO_CONVERGENCE = 2
RAFEAST_M0_TOO_SMALL = 3
RAFEAST_ERR_INVALID_ARG = -1
RAFEAST_ERR_NOT_SYMMETRIC = -2
RAFEAST_ERR_CUDA = -3
RAFEAST_ERR_COCG_BREAKDOWN = -4
RAFEAST_ERR_TIMEOUT = -5
RAFEAST_ERR_OUT_OF_MEMORY = -6
RAFEAST_ERR_NOT_READY = -7
RAFEAST_ERR_CHOLESKY = -8
RAFEAST_ERR_NO_DEVICE = -9
RAFEAST_ERR_EXCHANGE = -10

RAFEAST_FP64 = 0
RAFEAST_MIXED = 1
RAFEAST_FORM_DIRECT = 0
RAFEAST_FORM_CORRECTION = 1
RAFEAST_START_RANDOM = 0
RAFEAST_START_SUBSPACE = 1
RAFEAST_SHARD_COLUMNS = 0
RAFEAST_SHARD_SHIFTS = 1
RAFEAST_CREATE_NO_REORDER = 1
RAFEAST_CREATE_FORCE_REORDER = 2
RAFEAST_CREATE_CHECK_SYMMETRY = 4
RAFEAST_CREATE_RCM = 8
RAFEAST_OPT_WARMSTART_MAP = 1
RAFEAST_OPT_CHUNK = 2
RAFEAST_OPT_AUTOTUNE = 3
RAFEAST_OPT_LANES = 4
RAFEAST_OPT_PROFILE = 5
RAFEAST_OPT_KERNEL = 6
RAFEAST_OPT_MAXNZ = 7
RAFEAST_OPT_WAIT_LIMIT = 8
RAFEAST_OPT_TEST_STALL = 9
RAFEAST_OPT_CPL = 10
RAFEAST_OPT_SOLVER = 11
RAFEAST_OPT_UPDATE = 12
RAFEAST_OPT_VALUES_FREE = 13
RAFEAST_OPT_TILED = 14
RAFEAST_OPT_TILE_CB = 15
RAFEAST_OPT_DENSE = 16
RAFEAST_OPT_DEFER = 17

EXPORTS = [
    "rafeast_create", "rafeast_destroy", "rafeast_status_string", "rafeast_set_option",
    "rafeast_matrix_info", "rafeast_quadrature", "rafeast_philox", "rafeast_draw_omega",
    "rafeast_spmm", "rafeast_shifted_spmm", "rafeast_filter", "rafeast_orthonormalize",
    "rafeast_rayleigh_ritz", "rafeast_warmstart", "rafeast_set_subspace",
    "rafeast_get_subspace", "rafeast_solve", "rafeast_solve_batched", "rafeast_profile",
    "rafeast_last_error", "rafeast_profile_history", "rafeast_gram",
    "rafeast_gram_noalloc", "rafeast_shard_range", "rafeast_partition_instances",
    "rafeast_solve_sharded", "rafeast_block_product",
]

# int (*rafeast_sum_fn)(void* ctx, double* buf, int64_t count)
SUM_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64)


class RafeastParams(C.Structure):
    _fields_ = [("lmin", C.c_double), ("lmax", C.c_double), ("m0", C.c_int32),
                ("nc", C.c_int32), ("ellipse_ratio", C.c_double), ("solve_tol", C.c_double),
                ("outer_tol", C.c_double), ("max_outer", C.c_int32), ("max_inner", C.c_int32),
                ("precision", C.c_int32), ("solve_form", C.c_int32), ("start", C.c_int32),
                ("reserved", C.c_int32), ("seed", C.c_uint64)]


class RafeastInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer_iters", C.c_int32),
                ("cocg_iters_total", C.c_int32), ("cocg_min_last", C.c_int32),
                ("cocg_max_last", C.c_int32), ("cholqr_shifted", C.c_int32),
                ("kernel_launches", C.c_int32), ("spmm_launches", C.c_int32),
                ("max_resid", C.c_double), ("t_warmstart_ms", C.c_double),
                ("t_filter_ms", C.c_double), ("t_orth_ms", C.c_double),
                ("t_rr_ms", C.c_double), ("t_total_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RafeastError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {status_string(code)} ({code})")
        self.code = code


_lib = None


def load():
    """Load librafeast.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2512_01257_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    P, I, I64, U64, D, U32 = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double, C.c_uint32
    sig = {
        "rafeast_create": (I, [C.POINTER(P), I64, I64, P, P, P, D, I, P, U32]),
        "rafeast_destroy": (None, [P]),
        "rafeast_status_string": (C.c_char_p, [I]),
        "rafeast_last_error": (C.c_char_p, []),
        "rafeast_set_option": (I, [P, I, I64]),
        "rafeast_profile": (I, [P, I, P]),
        "rafeast_profile_history": (I, [P, I, P, P, P]),
        "rafeast_matrix_info": (I, [P, C.POINTER(I64), C.POINTER(I), C.POINTER(D),
                                    C.POINTER(D), C.POINTER(D)]),
        "rafeast_quadrature": (I, [D, D, I, D, P, P]),
        "rafeast_philox": (I, [U64, U64, I64, P, P]),
        "rafeast_draw_omega": (I, [P, U64, I, P]),
        "rafeast_spmm": (I, [P, I, D, D, P, P, I]),
        "rafeast_shifted_spmm": (I, [P, I, P, I, P, P, I]),
        "rafeast_filter": (I, [P, C.POINTER(RafeastParams), P, P, P, C.POINTER(RafeastInfo)]),
        "rafeast_orthonormalize": (I, [P, I, P, P]),
        "rafeast_rayleigh_ritz": (I, [P, I, P, P, P]),
        "rafeast_gram": (I, [P, I, P, P, P]),
        "rafeast_block_product": (I, [P, I, P, P, I, P]),
        "rafeast_gram_noalloc": (I, [P, P, I64, I, P, P]),
        "rafeast_warmstart": (I, [P, D, D, I, I, I, U64]),
        "rafeast_set_subspace": (I, [P, P, I, I]),
        "rafeast_get_subspace": (I, [P, P, P, I, I]),
        "rafeast_solve": (I, [P, C.POINTER(RafeastParams), C.POINTER(I), P, P, P, I,
                              C.POINTER(RafeastInfo)]),
        "rafeast_solve_batched": (I, [I, P, C.POINTER(RafeastParams), P, P, P, P, I,
                                      C.POINTER(RafeastInfo), P]),
        "rafeast_shard_range": (I, [I, I, I, I, I, C.POINTER(I), C.POINTER(I)]),
        "rafeast_partition_instances": (I, [I, P, I, P]),
        "rafeast_solve_sharded": (I, [P, C.POINTER(RafeastParams), I, I, I, SUM_FN, P,
                                      C.POINTER(I), P, P, P, I, C.POINTER(RafeastInfo)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().rafeast_status_string(int(code)).decode()


rafeast_status_string = status_string


def _check(code, where, ok=(RAFEAST_OK,)):
    if code not in ok:
        detail = load().rafeast_last_error().decode()
        err = RafeastError(code, where + (f" [{detail}]" if detail and code == RAFEAST_ERR_CUDA else ""))
        raise err
    return code


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(C.c_void_p)
    raise TypeError(type(x))


def _on_device(x) -> int:
    return int(hasattr(x, "is_cuda") and x.is_cuda)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def make_params(lmin, lmax, m0, nc, e=1.0, solve_tol=1e-10, outer_tol=1e-10, max_outer=20,
                max_inner=20000, precision=RAFEAST_FP64, solve_form=RAFEAST_FORM_CORRECTION,
                start=RAFEAST_START_RANDOM, seed=0) -> RafeastParams:
    return RafeastParams(lmin, lmax, m0, nc, e, solve_tol, outer_tol, max_outer, max_inner,
                         precision, solve_form, start, 0, seed)


# ---- entry points -------------------------------------------------------------

def rafeast_create(row_ptr, col_idx, values, diag_shift=0.0, n=None, stream=None, flags=0):
    """Create a handle for A = L + diag_shift I; inputs are numpy arrays (host)
    or torch CUDA tensors (int32, int32, float64)."""
    lib = load()
    dev = _on_device(row_ptr)
    if not dev:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float64)
    nn = (row_ptr.shape[0] - 1) if n is None else n
    nnz = col_idx.shape[0]
    h = C.c_void_p()
    rc = lib.rafeast_create(C.byref(h), nn, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                            float(diag_shift), dev, _stream(stream), flags)
    _check(rc, "rafeast_create")
    return h


def rafeast_destroy(h):
    load().rafeast_destroy(h)


def rafeast_set_option(h, key, value):
    return _check(load().rafeast_set_option(h, key, value), "rafeast_set_option")


def rafeast_profile(h, reset=True):
    """COCG kernel timing gathered with RAFEAST_OPT_PROFILE on."""
    out = np.zeros(8)
    _check(load().rafeast_profile(h, int(reset), _ptr(out)), "rafeast_profile")
    return dict(dots_launches=out[0], dots_ms=out[1], dots_bytes=out[2],
                update_launches=out[3], update_ms=out[4], update_bytes=out[5],
                dots_shape=int(out[6]), update_shape=int(out[7]))


def rafeast_profile_history(h):
    """(active columns, worst relative residual, [dot ms, update ms]) per
    COCG step of the last profiled solve."""
    lib = load()
    n = lib.rafeast_profile_history(h, 0, None, None, None)
    _check(min(n, 0), "rafeast_profile_history")
    cols = np.zeros(n, dtype=np.int32)
    res = np.zeros(n)
    ms = np.zeros((n, 2))
    lib.rafeast_profile_history(h, n, _ptr(cols), _ptr(res), _ptr(ms))
    return cols, res, ms


def rafeast_matrix_info(h):
    n, r, n1, lo, hi = C.c_int64(), C.c_int(), C.c_double(), C.c_double(), C.c_double()
    _check(load().rafeast_matrix_info(h, C.byref(n), C.byref(r), C.byref(n1), C.byref(lo),
                                      C.byref(hi)), "rafeast_matrix_info")
    return dict(n=n.value, reordered=bool(r.value), order=int(r.value), norm1=n1.value,
                gersh_lo=lo.value, gersh_hi=hi.value)


def rafeast_quadrature(lmin, lmax, nc, e=1.0):
    z = np.zeros(2 * nc)
    w = np.zeros(2 * nc)
    _check(load().rafeast_quadrature(lmin, lmax, nc, e, _ptr(z), _ptr(w)), "rafeast_quadrature")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def rafeast_philox(seed, first_block, nblocks, words, stream=None):
    """words: torch CUDA int64/uint64 tensor of 4*nblocks entries."""
    return _check(load().rafeast_philox(C.c_uint64(seed), C.c_uint64(first_block), nblocks,
                                        _ptr(words), _stream(stream)), "rafeast_philox")


def rafeast_draw_omega(h, seed, k, omega):
    """omega: torch CUDA float64 tensor of shape (k, n) (column-major n x k)."""
    return _check(load().rafeast_draw_omega(h, C.c_uint64(seed), k, _ptr(omega)),
                  "rafeast_draw_omega")


def rafeast_spmm(h, k, alpha, beta, X, Y, precision=RAFEAST_FP64):
    return _check(load().rafeast_spmm(h, k, alpha, beta, _ptr(X), _ptr(Y), precision),
                  "rafeast_spmm")


def rafeast_shifted_spmm(h, nc, z, m, P, W, precision=RAFEAST_FP64):
    """z: complex array of nc shifts; P, W: torch CUDA float64 tensors holding
    n*m*nc complex values as (re, im) pairs, entry (i, col, j) at
    2*((col*nc + j)*n + i)."""
    zz = np.zeros(2 * nc)
    zz[0::2] = np.real(z)
    zz[1::2] = np.imag(z)
    return _check(load().rafeast_shifted_spmm(h, nc, _ptr(zz), m, _ptr(P), _ptr(W), precision),
                  "rafeast_shifted_spmm")


def rafeast_filter(h, params, Q, theta, Qt):
    info = RafeastInfo()
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    rc = load().rafeast_filter(h, C.byref(params), _ptr(Q), _ptr(th), _ptr(Qt), C.byref(info))
    _check(rc, "rafeast_filter")
    return info


def rafeast_orthonormalize(h, m, Q, want_r=False):
    R = np.zeros((m, m)) if want_r else None
    _check(load().rafeast_orthonormalize(h, m, _ptr(Q), _ptr(R)), "rafeast_orthonormalize")
    return None if R is None else R.T.copy()  # column-major -> (row, col)


def rafeast_gram(h, m, X, Y, G):
    """G = X^T Y; X, Y CUDA tensors (m, n) (column-major n x m), G CUDA (m, m)
    holding the column-major m x m result (G[b, a] = entry (a, b))."""
    return _check(load().rafeast_gram(h, m, _ptr(X), _ptr(Y), _ptr(G)), "rafeast_gram")


def rafeast_block_product(h, m, X, M, mo, Y):
    """Y = X M: X (m, n), M (mo, m) and Y (mo, n) CUDA tensors (column-major
    n x m, m x mo and n x mo blocks)."""
    _check(load().rafeast_block_product(h, int(m), _ptr(X), _ptr(M), int(mo), _ptr(Y)),
           "rafeast_block_product")


def rafeast_gram_noalloc(X, Y, n, m, G, stream=None):
    """Allocation-free G = X^T Y (same layouts as rafeast_gram, no handle).
    Enqueues on ``stream`` (default: torch's current stream) and returns."""
    return _check(load().rafeast_gram_noalloc(_ptr(X), _ptr(Y), n, m, _ptr(G), _stream(stream)),
                  "rafeast_gram_noalloc")


def rafeast_rayleigh_ritz(h, m, Q):
    theta = np.zeros(m)
    res = np.zeros(m)
    _check(load().rafeast_rayleigh_ritz(h, m, _ptr(Q), _ptr(theta), _ptr(res)),
           "rafeast_rayleigh_ritz")
    return theta, res


def rafeast_warmstart(h, lmin, lmax, m0, p, q, seed):
    return _check(load().rafeast_warmstart(h, lmin, lmax, m0, p, q, C.c_uint64(seed)),
                  "rafeast_warmstart")


def rafeast_set_subspace(h, Q0, m0):
    return _check(load().rafeast_set_subspace(h, _ptr(Q0), m0, _on_device(Q0)),
                  "rafeast_set_subspace")


def rafeast_get_subspace(h, Q, m0):
    theta = np.zeros(m0)
    _check(load().rafeast_get_subspace(h, _ptr(Q), _ptr(theta), m0, _on_device(Q)),
           "rafeast_get_subspace")
    return theta


def rafeast_solve(h, params, evals, evecs=None, resid=None):
    """Outputs are numpy arrays (host) or torch CUDA tensors (device), all of
    the same kind. Returns (status, m_found, info)."""
    info = RafeastInfo()
    mf = C.c_int()
    dev = _on_device(evals)
    rc = load().rafeast_solve(h, C.byref(params), C.byref(mf), _ptr(evals), _ptr(evecs),
                              _ptr(resid), dev, C.byref(info))
    _check(rc, "rafeast_solve", ok=(0, 1, 2, 3))
    return rc, mf.value, info


def rafeast_solve_batched(handles, params, evals, evecs=None, resid=None):
    n = len(handles)
    H = (C.c_void_p * n)(*[h.value for h in handles])
    Pa = (RafeastParams * n)(*params)
    MF = (C.c_int * n)()
    ST = (C.c_int * n)()
    INF = (RafeastInfo * n)()
    dev = _on_device(evals[0])
    E = (C.c_void_p * n)(*[_ptr(e).value for e in evals])
    V = None if evecs is None else (C.c_void_p * n)(*[_ptr(v).value for v in evecs])
    R = None if resid is None else (C.c_void_p * n)(*[_ptr(r).value for r in resid])
    rc = load().rafeast_solve_batched(n, H, Pa, MF, E, V, R, dev, INF, ST)
    _check(rc, "rafeast_solve_batched")
    return list(ST), list(MF), list(INF)


def rafeast_shard_range(mode, m0, nc, rank, world):
    """(lo, hi): the columns (RAFEAST_SHARD_COLUMNS) or quadrature nodes
    (RAFEAST_SHARD_SHIFTS) that rank filters in a sharded solve."""
    lo, hi = C.c_int(), C.c_int()
    _check(load().rafeast_shard_range(int(mode), int(m0), int(nc), int(rank), int(world),
                                      C.byref(lo), C.byref(hi)), "rafeast_shard_range")
    return lo.value, hi.value


def rafeast_partition_instances(costs, world):
    """owner[i]: the rank that solves problem i (longest first, least loaded)."""
    cost = np.ascontiguousarray(costs, dtype=np.int64)
    owner = np.zeros(len(cost), dtype=np.int32)
    _check(load().rafeast_partition_instances(len(cost), _ptr(cost), int(world), _ptr(owner)),
           "rafeast_partition_instances")
    return owner


class _DeviceView:
    """A (count,) float64 view of device memory for torch.as_tensor."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                         "data": (int(ptr), False), "strides": None,
                                         "version": 2}


def device_tensor(ptr, count):
    """torch float64 tensor over count doubles of device memory at ptr (no copy)."""
    import torch
    return torch.as_tensor(_DeviceView(ptr, count), device="cuda")


def allreduce_sum(group=None):
    """Sum over the ranks of a torch.distributed group (NCCL, or gloo with
    CUDA tensors) for rafeast_solve_sharded: an all-reduce of the block in
    place, finished before the call returns."""
    import torch
    import torch.distributed as dist

    def fn(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        if t.is_cuda:
            torch.cuda.current_stream(t.device).synchronize()
    return fn


def rafeast_solve_sharded(h, params, mode, rank, world, sum_fn, evals, evecs=None, resid=None):
    """rafeast_solve on rank `rank` of `world`. sum_fn(t) receives a torch
    float64 CUDA tensor viewing the library's block and must leave in it the
    sum over ranks (e.g. allreduce_sum()). An exception in sum_fn fails the
    solve and is raised here. Returns (status, m_found, info)."""
    info = RafeastInfo()
    mf = C.c_int()
    dev = _on_device(evals)
    failure = []

    def cb(_ctx, buf, count):
        try:
            sum_fn(device_tensor(buf, count))
            return 0
        except BaseException as e:  # noqa: BLE001 (reported after the call)
            failure.append(e)
            return 1
    fn = SUM_FN(cb) if sum_fn is not None else SUM_FN()
    rc = load().rafeast_solve_sharded(h, C.byref(params), int(mode), int(rank), int(world), fn,
                                      None, C.byref(mf), _ptr(evals), _ptr(evecs), _ptr(resid),
                                      dev, C.byref(info))
    if failure:
        raise RafeastError(rc, "rafeast_solve_sharded: sum callback") from failure[0]
    _check(rc, "rafeast_solve_sharded", ok=(0, 1, 2, 3))
    return rc, mf.value, info
