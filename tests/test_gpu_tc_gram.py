"""Tensor-core FP64 Gram matrix (FP64 values split into exact BF16 digits,
tcgen05 products, integer accumulation) against an exact reference.

The Gram matrices of the Cholesky-QR and Rayleigh-Ritz steps (Algorithm 1)
are formed this way by default. The reference is the same contraction in
extended precision on the host (numpy longdouble, then rounded); the gate is
eight units of 2^-53 times sum_k |x_ka y_kb| (the FP64 pipe's own Gram, run
beside it, is held to the classical n units), on inputs that stress the
scaling: ragged row counts (one CTA's rows, many CTAs, a partial 32-row
sub-chunk, more than one 128-row exact chunk), every column-count edge
(1, a multiple of 16, odd, 80 = two column blocks, 116, 128), X = Y (one
digit split feeds both operands), a zero column, columns whose magnitudes
span 10^-150 .. 10^150, and columns with a single value far above the rest.
For the latter the splitting's own bound applies: values are written to
2^-55 of their column's largest value over the rows one CTA owns, so a
single spike coarsens its neighbours; the test adds that bound.
"""
import numpy as np
import pytest

from gpu_util import colmajor_dev
from workloads import graphs as G

pytestmark = pytest.mark.gpu


def _inputs(n, m, kind, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, m))
    y = rng.standard_normal((n, m))
    if kind == "scaled":
        sx = 10.0 ** rng.uniform(-150, 150, m)
        sy = 10.0 ** rng.uniform(-150, 150, m)
        x *= sx
        y *= sy
    elif kind == "spikes":
        x[rng.integers(0, n, m), np.arange(m)] *= 1e6
        y[rng.integers(0, n, m), np.arange(m)] *= -1e5
        x[:, 0] = 0.0
    return x, y


def _reference(x, y):
    xl, yl = x.astype(np.longdouble), y.astype(np.longdouble)
    return (xl.T @ yl).astype(np.float64), np.abs(x).T @ np.abs(y)


def _split_bound(x, y, parts):
    """The splitting's error bound: a CTA owns rows [n c / P, n (c+1) / P)
    and writes each value of a column to 2^-55 of that column's largest
    value over its rows, so a product errs by at most 2^-54 Mx_a My_b per
    row (M: the column maxima over the CTA's rows)."""
    n = x.shape[0]
    bound = np.zeros((x.shape[1], y.shape[1]))
    for c in range(parts):
        lo, hi = n * c // parts, n * (c + 1) // parts
        if hi > lo:
            mx = np.abs(x[lo:hi]).max(axis=0)
            my = np.abs(y[lo:hi]).max(axis=0)
            bound += (hi - lo) * np.outer(mx, my)
    return 2.0 ** -53 * bound


@pytest.mark.parametrize("n", [5, 100, 2867])
@pytest.mark.parametrize("m", [1, 16, 33, 80, 116, 128])
@pytest.mark.parametrize("kind", ["gauss", "scaled", "spikes"])
def test_tensor_core_gram_is_fp64_accurate(lib, n, m, kind):
    import torch
    parts = torch.cuda.get_device_properties(0).multi_processor_count  # CTAs over rows
    lap = G.path(n)
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, 0.0)
    try:
        for same in (False, True):
            x, y = _inputs(n, m, kind, 100 * n + m)
            if same:
                y = x
            exp, absprod = _reference(x, y)
            X = colmajor_dev(x)
            Y = X if same else colmajor_dev(y)
            for dense in (0, 1):  # tensor cores, FP64 pipe
                lib.rafeast_set_option(h, lib.RAFEAST_OPT_DENSE, dense)
                Gd = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")
                lib.rafeast_gram(h, m, X, Y, Gd)  # G = X^T Y, column-major
                got = Gd.cpu().numpy().T
                err = np.abs(got - exp)
                # tensor cores: the digit products are summed exactly, so
                # the error is the splitting's, a few units of 2^-53; the
                # FP64 pipe sums in floating point (the classical n u bound)
                units = 8.0 if dense == 0 else 8.0 + n
                tol = units * 2.0 ** -53 * absprod + 1e-300
                if dense == 0 and kind == "spikes":
                    tol += _split_bound(x, y, parts)
                assert np.all(err <= tol), (same, dense, float(np.max(err / tol)))
    finally:
        lib.rafeast_destroy(h)
