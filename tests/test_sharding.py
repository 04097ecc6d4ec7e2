"""Sharding over ranks, on CPU: the shares rafeast_shard_range hands out
(columns of Q in whole pairs, or quadrature nodes), the longest-first
instance partition (checked against brute force on small cases, with
Graham's bound), and the sharded FEAST loop on a world-size-2 gloo group:
each rank filters its share with the oracle, the binding's all-reduce adds
the partial blocks, and the result equals the single-rank oracle FEAST."""
import itertools
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    from paper_2512_01257_gb300 import build, rafeast
    if not os.path.exists(rafeast.LIB_PATH):
        build.build()
    return rafeast


@pytest.mark.parametrize("mode", [0, 1])
def test_shard_ranges_tile_the_work(R, mode):
    for total in list(range(1, 21)) + [42, 63, 80, 96, 128]:
        for world in range(1, 10):
            m0, nc = (total, 4) if mode == R.RAFEAST_SHARD_COLUMNS else (8, min(total, 16))
            n_units = m0 if mode == R.RAFEAST_SHARD_COLUMNS else nc
            rng = [R.rafeast_shard_range(mode, m0, nc, r, world) for r in range(world)]
            # in rank order, back to back, covering every unit once
            assert rng[0][0] == 0 and rng[-1][1] == n_units
            for (a, b), (c, d) in zip(rng, rng[1:]):
                assert b == c
            assert all(lo <= hi for lo, hi in rng)
            if mode == R.RAFEAST_SHARD_COLUMNS:
                # whole column pairs: every share starts on an even column,
                # and the pair counts differ by at most one
                assert all(lo % 2 == 0 for lo, _ in rng)
                pairs = [((hi - lo) + 1) // 2 for lo, hi in rng]
                assert max(pairs) - min(pairs) <= 1
                assert sum(pairs) == (m0 + 1) // 2
            else:
                sizes = [hi - lo for lo, hi in rng]
                assert max(sizes) - min(sizes) <= 1


def test_shard_range_rejects_bad_arguments(R):
    for args in [(2, 8, 4, 0, 1), (0, 8, 4, 1, 1), (0, 8, 4, -1, 2), (0, 0, 4, 0, 1),
                 (1, 8, 0, 0, 1), (0, 8, 4, 0, 0)]:
        with pytest.raises(R.RafeastError):
            R.rafeast_shard_range(*args)


def _makespan(costs, owner, world):
    load = [0] * world
    for c, o in zip(costs, owner):
        load[o] += c
    return max(load)


def test_partition_instances_longest_first(R):
    rng = np.random.default_rng(7)
    for trial in range(60):
        count = int(rng.integers(1, 8))
        world = int(rng.integers(2, 4))
        costs = [int(c) for c in rng.integers(1, 1000, count)]
        owner = R.rafeast_partition_instances(costs, world)
        assert owner.shape == (count,) and owner.min() >= 0 and owner.max() < world
        # the same owners on every call (every rank computes them itself)
        assert np.array_equal(owner, R.rafeast_partition_instances(costs, world))
        got = _makespan(costs, owner, world)
        best = min(_makespan(costs, o, world)
                   for o in itertools.product(range(world), repeat=count))
        # Graham (1969): longest processing time first is within
        # 4/3 - 1/(3m) of the optimum on m machines
        assert got <= (4.0 / 3.0 - 1.0 / (3 * world)) * best + 1e-9
    # one problem per rank when there are enough ranks; empty input
    owner = R.rafeast_partition_instances([5, 9, 1], 4)
    assert sorted(owner.tolist()) == [0, 1, 2] and owner[1] == 0
    assert R.rafeast_partition_instances([], 3).shape == (0,)
    with pytest.raises(R.RafeastError):
        R.rafeast_partition_instances([1, -2], 2)
    with pytest.raises(R.RafeastError):
        R.rafeast_partition_instances([1, 2], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    sys.path.insert(0, ROOT)
    from workloads import graphs as G
    lap = G.grid2d(12, 15, 0.0)
    return lap.scipy()


def _sharded_feast(a, q0, lmin, lmax, nc, mode, rank, world, reduce_fn, R):
    """Phase 2 with the filter split over ranks: the oracle's filter on this
    rank's share, the partial blocks added by reduce_fn, then the same
    orthonormalisation, Rayleigh-Ritz and residual steps on every rank."""
    import torch
    from oracle import feast as OF
    from oracle import quadrature as OQ
    z, w = OQ.nodes(lmin, lmax, nc, 1.0)
    m0 = q0.shape[1]
    lo, hi = R.rafeast_shard_range(mode, m0, nc, rank, world)
    q, theta = q0, None
    norm_a = OF.one_norm(a)
    for it in range(1, 21):
        qt = np.zeros_like(q)
        if hi > lo:
            if mode == R.RAFEAST_SHARD_COLUMNS:
                qt[:, lo:hi], _ = OF.filter_apply(a, q[:, lo:hi], z, w, 1e-12, 5000, "direct")
            else:
                qt, _ = OF.filter_apply(a, q, z[lo:hi], w[lo:hi], 1e-12, 5000, "direct")
        t = torch.from_numpy(qt)
        reduce_fn(t)
        q = OF.orthonormalize(t.numpy())
        lam, q, aq = OF.rayleigh_ritz(a, q)
        res = OF.residuals(a, lam, q, aq, norm_a)
        inside = (lam >= lmin) & (lam <= lmax)
        flag = torch.tensor([1.0 if inside.any() and res[inside].max() <= 1e-10 else 0.0],
                            dtype=torch.float64)
        reduce_fn(flag)
        if flag.item() > world - 0.5:
            break
    return lam[inside], it, q


def _rank(rank, world, port, out, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from oracle import feast as OF
    from paper_2512_01257_gb300 import rafeast as R
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a = _problem()
    q0 = OF.random_start(a.shape[0], 12, 5)
    lam, it, q = _sharded_feast(a, q0, 0.0, 0.3, 4, mode, rank, world, R.allreduce_sum(), R)
    np.save(os.path.join(out, f"q{rank}.npy"), q)
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"evals": lam.tolist(), "iters": it}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", [0, 1])
def test_sharded_feast_two_gloo_ranks(R, tmp_path, mode):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from oracle import feast as OF
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path), mode), nprocs=2,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    qs = [np.load(tmp_path / f"q{r}.npy") for r in range(2)]
    # both ranks hold the same bits
    assert res[0] == res[1]
    assert np.array_equal(qs[0], qs[1])
    # and the single-rank oracle's result
    a = _problem()
    q0 = OF.random_start(a.shape[0], 12, 5)
    ref = OF.feast(a, 0.0, 0.3, q0, 4, 1.0, 1e-12, 1e-10, 20, 5000, "direct")
    assert ref.status == 0
    assert res[0]["iters"] == ref.outer_iters
    got = np.array(res[0]["evals"])
    assert got.shape == ref.evals.shape
    # columns: each column's solve is the single-rank one, and adding zeros
    # is exact; nodes: the quadrature sum is added in two parts (the
    # spectrum includes 0, so the error is absolute, against the interval)
    if mode == R.RAFEAST_SHARD_COLUMNS:
        assert np.array_equal(got, ref.evals)
    else:
        assert np.max(np.abs(got - ref.evals)) <= 1e-14
