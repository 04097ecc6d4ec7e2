"""rafeast_solve_sharded through the C-ABI on one GPU: the ranks of a world
of 2 or 3 run as host threads of one process, each with its own handle and
stream; their sum meets on a host barrier after every rank's stream is idle
(no kernel of one rank waits on another's). Checked: every rank ends with
the same bits, the eigenpairs match the single-rank solve and the stored
spectrum, world = 1 repeats rafeast_solve to the last bit, and a failing
sum fails the solve on every rank with RAFEAST_ERR_EXCHANGE, leaving the
handles usable."""
import threading

import numpy as np
import pytest

from oracle import metrics as M
from workloads import configs as CF

pytestmark = pytest.mark.gpu


class ThreadSum:
    """Sum over ranks run as threads: each adds all blocks in rank order."""

    def __init__(self, world, fail_rank=-1):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.bufs = [None] * world
        self.fail_rank = fail_rank
        self.calls = [0] * world

    def for_rank(self, r):
        import torch

        def fn(t):
            self.calls[r] += 1
            if r == self.fail_rank:
                self.bar.abort()
                raise RuntimeError("planted sum failure")
            self.bufs[r] = t
            self.bar.wait()
            s = self.bufs[0].clone()
            for q in range(1, self.world):
                s += self.bufs[q]
            torch.cuda.current_stream().synchronize()
            self.bar.wait()  # every rank has read every block
            t.copy_(s)
            torch.cuda.current_stream().synchronize()
        return fn


@pytest.fixture(scope="module")
def knn8k():
    lap = CF.CONFIGS["knn8k"].make()
    g = CF.load_golden()["knn8k"]
    assert g["checksum"] == lap.checksum()
    return lap, g


def _params(lib, g, prec, nc):
    cfg = CF.CONFIGS["knn8k"]
    p = lib.RAFEAST_FP64 if prec == "fp64" else lib.RAFEAST_MIXED
    return lib.make_params(g["lmin"], g["lmax"], cfg.m0, nc, 1.0, cfg.solve_tol, cfg.outer_tol,
                           cfg.max_outer, cfg.max_inner, p, lib.RAFEAST_FORM_CORRECTION,
                           lib.RAFEAST_START_SUBSPACE)


def _outputs(m0, n):
    return np.zeros(m0), np.zeros((m0, n)), np.zeros(m0)


def _run_ranks(lib, lap, g, prm, mode, world, fail_rank=-1):
    cfg = CF.CONFIGS["knn8k"]
    ts = ThreadSum(world, fail_rank)
    hs = [lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
          for _ in range(world)]
    out = [None] * world

    def rank(r):
        import torch
        torch.cuda.set_device(0)
        try:
            lib.rafeast_warmstart(hs[r], g["lmin"], g["lmax"], cfg.m0, cfg.p, cfg.q, cfg.seed)
            ev, vec, res = _outputs(cfg.m0, lap.n)
            st, mf, info = lib.rafeast_solve_sharded(hs[r], prm, mode, r, world,
                                                     ts.for_rank(r), ev, vec, res)
            out[r] = (st, mf, ev, vec, res, info.outer_iters)
        except Exception as e:  # noqa: BLE001 (checked by the caller)
            out[r] = e
    th = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return hs, out, ts


@pytest.mark.parametrize("mode,world,nc,prec", [
    ("columns", 2, 4, "mixed"), ("columns", 3, 4, "fp64"),
    ("shifts", 2, 4, "mixed"), ("shifts", 3, 2, "fp64"),   # one rank without a node
])
def test_sharded_matches_single_rank(lib, knn8k, mode, world, nc, prec):
    lap, g = knn8k
    cfg = CF.CONFIGS["knn8k"]
    m = lib.RAFEAST_SHARD_COLUMNS if mode == "columns" else lib.RAFEAST_SHARD_SHIFTS
    prm = _params(lib, g, prec, nc)
    hs, out, ts = _run_ranks(lib, lap, g, prm, m, world)
    try:
        for o in out:
            assert not isinstance(o, Exception), o
        st, mf, ev, vec, res, iters = out[0]
        assert st == lib.RAFEAST_OK and mf == 32
        for o in out[1:]:
            assert o[0] == st and o[1] == mf and o[5] == iters
            assert np.array_equal(o[2], ev) and np.array_equal(o[3], vec)
            assert np.array_equal(o[4], res)
        # two sums (block, stop flag) per outer iteration on every rank
        assert ts.calls == [2 * iters] * world
        # the same problem on one rank
        h1 = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
        try:
            lib.rafeast_warmstart(h1, g["lmin"], g["lmax"], cfg.m0, cfg.p, cfg.q, cfg.seed)
            e1, v1, r1 = _outputs(cfg.m0, lap.n)
            st1, mf1, _ = lib.rafeast_solve(h1, prm, e1, v1, r1)
        finally:
            lib.rafeast_destroy(h1)
        assert st1 == lib.RAFEAST_OK and mf1 == mf
        tol_e, tol_v = (1e-10, 1e-8) if prec == "fp64" else (1e-8, 1e-6)
        assert M.eig_relerr(ev[:mf], e1[:mf1]) <= tol_e
        assert M.eig_relerr(ev[:mf], g["evals"]) <= tol_e
        assert M.sin_theta(vec[:mf].T, v1[:mf1].T) <= tol_v
        assert np.all(res[:mf] <= cfg.outer_tol)
    finally:
        for h in hs:
            lib.rafeast_destroy(h)


@pytest.mark.parametrize("mode", ["columns", "shifts"])
def test_world_one_is_rafeast_solve(lib, knn8k, mode):
    lap, g = knn8k
    cfg = CF.CONFIGS["knn8k"]
    m = lib.RAFEAST_SHARD_COLUMNS if mode == "columns" else lib.RAFEAST_SHARD_SHIFTS
    prm = _params(lib, g, "mixed", 4)
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
    try:
        # (the first solve runs the autotuner's candidate shapes for its first
        # COCG steps; solves after it repeat to the last bit)
        outs = []
        for sharded in (False, False, True, False):
            lib.rafeast_warmstart(h, g["lmin"], g["lmax"], cfg.m0, cfg.p, cfg.q, cfg.seed)
            ev, vec, res = _outputs(cfg.m0, lap.n)
            if sharded:
                st, mf, _ = lib.rafeast_solve_sharded(h, prm, m, 0, 1, None, ev, vec, res)
            else:
                st, mf, _ = lib.rafeast_solve(h, prm, ev, vec, res)
            assert st == lib.RAFEAST_OK
            outs.append((ev, vec, res))
        for a, b in zip(outs[1], outs[2]):
            assert np.array_equal(a, b)
        for a, b in zip(outs[1], outs[3]):
            assert np.array_equal(a, b)
    finally:
        lib.rafeast_destroy(h)


def test_failed_sum_fails_every_rank(lib, knn8k):
    lap, g = knn8k
    cfg = CF.CONFIGS["knn8k"]
    prm = _params(lib, g, "mixed", 4)
    hs, out, ts = _run_ranks(lib, lap, g, prm, lib.RAFEAST_SHARD_COLUMNS, 2, fail_rank=1)
    try:
        for o in out:
            assert isinstance(o, lib.RafeastError), o
            assert o.code == lib.RAFEAST_ERR_EXCHANGE
        # the handles still solve
        lib.rafeast_warmstart(hs[0], g["lmin"], g["lmax"], cfg.m0, cfg.p, cfg.q, cfg.seed)
        ev, vec, res = _outputs(cfg.m0, lap.n)
        st, mf, _ = lib.rafeast_solve(hs[0], prm, ev, vec, res)
        assert st == lib.RAFEAST_OK and mf == 32
    finally:
        for h in hs:
            lib.rafeast_destroy(h)


def test_sharded_argument_checks(lib, knn8k):
    lap, g = knn8k
    prm = _params(lib, g, "mixed", 4)
    h = lib.rafeast_create(lap.row_ptr, lap.col_idx, lap.values, lap.shift)
    try:
        ev, vec, res = _outputs(prm.m0, lap.n)
        for mode, rank, world, fn in [(2, 0, 1, None), (0, 2, 2, lambda t: None),
                                      (0, -1, 2, lambda t: None), (0, 0, 0, None),
                                      (0, 0, 2, None)]:
            with pytest.raises(lib.RafeastError) as e:
                lib.rafeast_solve_sharded(h, prm, mode, rank, world, fn, ev, vec, res)
            assert e.value.code == lib.RAFEAST_ERR_INVALID_ARG
    finally:
        lib.rafeast_destroy(h)
