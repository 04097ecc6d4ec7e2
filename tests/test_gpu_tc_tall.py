"""Tensor-core FP64 tall block product Y = X M (FP64 values split into exact
BF16 digits, tcgen05 products, exact integer levels) against an exact
reference, through rafeast_block_product.

The products X R^{-1} of the Cholesky-QR passes and X (R^{-1} V) of the
Rayleigh-Ritz step (Algorithm 1) are formed this way by default. The
reference is the same product in extended precision on the host (numpy
longdouble); the gate is the splitting's bound: each CTA scales column a of
X by the power of two above its largest magnitude over the CTA's rows and M's
row a by the same power, then writes every value of a row of X (of a column
of M) to 2^-55 of that row's (column's) largest scaled value; the digit
levels are exact, and one rounding to FP64 ends it. The FP64 pipe's kernel,
run beside it, is held to the classical m units of 2^-53 of |X| |M|. Inputs:
ragged row counts (one CTA's rows, a partial 128-row block, many blocks), m
and mo at every edge (1, 16, 33, 80 = two column blocks, 100 x 80 as in the
warmstart, 128), columns of X spanning 10^-150 .. 10^150, a zero column and
a zero row, an upper-triangular M, and NaN propagation."""
import numpy as np
import pytest

from gpu_util import colmajor_dev
from workloads import graphs as G

pytestmark = pytest.mark.gpu


def _parts(n, mo, sms):
    """The kernel's row partition: column blocks of nb <= 64 (a multiple of
    16), the SMs shared out over them, row ranges [n c / P, n (c+1) / P)."""
    nblk = -(-mo // 64)
    nb = -(-mo // nblk)
    nb = -(-nb // 16) * 16
    nbx = -(-mo // nb)
    parts = max(1, sms // nbx)
    blocks = -(-n // 128)
    return max(1, min(parts, blocks))


def _split_bound(x, mm, parts):
    """2^-55 (rowmax'_r sum_a |M'_ab| + colmax'_b sum_a |x'_ra|) per entry,
    with the CTA's column scaling x' = x / s_a, M' = s_a M."""
    n = x.shape[0]
    out = np.zeros((n, mm.shape[1]))
    for c in range(parts):
        lo, hi = n * c // parts, n * (c + 1) // parts
        if hi <= lo:
            continue
        xs = x[lo:hi]
        cm = np.abs(xs).max(axis=0)
        s = np.where(cm > 0, np.ldexp(1.0, np.frexp(cm)[1]), 1.0)
        xp = np.abs(xs) / s
        mp = np.abs(mm) * s[:, None]
        rowmax = xp.max(axis=1)
        colmax = mp.max(axis=0)
        out[lo:hi] = 2.0 ** -55 * (np.outer(rowmax, mp.sum(axis=0)) + np.outer(xp.sum(axis=1), colmax))
    return out


def _inputs(n, m, mo, kind, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, m))
    mm = rng.standard_normal((m, mo))
    if kind == "scaled":
        x *= 10.0 ** rng.uniform(-150, 150, m)
        mm /= 10.0 ** rng.uniform(-100, 100, m)[:, None]
        x[:, m // 2] = 0.0
        x[n // 2, :] = 0.0
    elif kind == "upper":
        mm = np.triu(rng.standard_normal((m, mo)))
    return x, mm


@pytest.mark.parametrize("n", [7, 300, 4099])
@pytest.mark.parametrize("m,mo", [(1, 1), (16, 16), (33, 17), (80, 80), (100, 80), (128, 128)])
@pytest.mark.parametrize("kind", ["gauss", "scaled", "upper"])
def test_tensor_core_block_product_is_fp64_accurate(lib, n, m, mo, kind):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lap = G.path(n)
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, 0.0)
    try:
        x, mm = _inputs(n, m, mo, kind, 1000 * n + 10 * m + mo)
        exp = (x.astype(np.longdouble) @ mm.astype(np.longdouble)).astype(np.float64)
        absprod = np.abs(x) @ np.abs(mm)
        X = colmajor_dev(x)
        Md = colmajor_dev(mm)  # column-major m x mo
        for dense in (0, 1):  # tensor cores, FP64 pipe
            lib.rafeast_set_option(h, lib.RAFEAST_OPT_DENSE, dense)
            Yd = torch.full((mo, n), float("nan"), dtype=torch.float64, device="cuda")
            lib.rafeast_block_product(h, m, X, Md, mo, Yd)
            got = Yd.cpu().numpy().T
            err = np.abs(got - exp)
            if dense == 0:
                tol = 2.0 * _split_bound(x, mm, _parts(n, mo, sms)) + 2.0 ** -52 * np.abs(exp)
            else:
                tol = (m + 2) * 2.0 ** -53 * absprod
            tol += 1e-300
            assert np.all(np.isfinite(got))
            assert np.all(err <= tol), (dense, float(np.max(err / tol)))
    finally:
        lib.rafeast_destroy(h)


def test_block_product_nan_rows_and_columns(lib):
    import torch
    n, m, mo = 500, 24, 40
    lap = G.path(n)
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, 0.0)
    try:
        rng = np.random.default_rng(5)
        x = rng.standard_normal((n, m))
        mm = rng.standard_normal((m, mo))
        x[17, 3] = np.nan
        x[230, 0] = np.inf
        mm[5, 11] = np.nan
        Yd = torch.zeros((mo, n), dtype=torch.float64, device="cuda")
        lib.rafeast_block_product(h, m, colmajor_dev(x), colmajor_dev(mm), mo, Yd)
        got = Yd.cpu().numpy().T
        bad_r = np.zeros(n, bool)
        bad_r[[17, 230]] = True
        bad_c = np.zeros(mo, bool)
        bad_c[11] = True
        assert np.all(np.isnan(got[bad_r, :]))
        assert np.all(np.isnan(got[:, bad_c]))
        ok = got[~bad_r][:, ~bad_c]
        exp = (x[~bad_r] @ mm)[:, ~bad_c]
        assert np.all(np.isfinite(ok))
        assert np.allclose(ok, exp, rtol=1e-13, atol=1e-13)
        with pytest.raises(lib.RafeastError):
            lib.rafeast_block_product(h, 0, colmajor_dev(x), colmajor_dev(mm), mo, Yd)
        with pytest.raises(lib.RafeastError):
            lib.rafeast_block_product(h, m, colmajor_dev(x), colmajor_dev(mm), 129, Yd)
    finally:
        lib.rafeast_destroy(h)
