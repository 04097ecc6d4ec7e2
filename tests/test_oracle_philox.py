"""Pins of the oracle's Omega generator (Algorithm 2, "Draw Omega").

The Philox-4x64-10 rounds are checked word for word against
``numpy.random.Philox`` (the same published generator, a library routine).
numpy increments its 256-bit counter before producing each block, so its
first block for counter state C is the block for C + 1. The Gaussian
transform is checked by distribution (Kolmogorov-Smirnov) and by the block
layout the module docstring states.
"""
import numpy as np
import pytest
import scipy.stats

from oracle import philox as P


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 17])
def test_blocks_match_numpy_philox(seed):
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64))
    raw = bg.random_raw(4 * 6)
    mine = P.philox_blocks(np.arange(1, 7, dtype=np.uint64), seed).ravel()
    assert np.array_equal(raw, mine)


def test_counter_wrap_matches_numpy():
    ones = np.array([2**64 - 1] * 4, dtype=np.uint64)
    bg = np.random.Philox(key=ones[:2], counter=ones)
    raw = bg.random_raw(4)
    mine = P.philox4x64_10((0, 0, 0, 0), (2**64 - 1, 2**64 - 1))
    assert [int(v) for v in raw] == list(mine)


def test_vectorised_equals_scalar():
    seed = 987654321
    blocks = P.philox_blocks(np.arange(0, 50, dtype=np.uint64), seed)
    for b in range(50):
        assert tuple(int(v) for v in blocks[b]) == P.philox4x64_10((b, 0, 0, 0), (seed, 0))


def test_uniform_range():
    u = P.uniforms(np.array([0, 2**64 - 1], dtype=np.uint64))
    assert u[0] == 2.0 ** -53 and u[1] == 1.0


def test_gaussian_layout():
    n, k, seed = 37, 5, 3
    om = P.gaussian_matrix(n, k, seed)
    words = P.philox_words(n, k, seed)
    u = P.uniforms(words)
    # entry (i, c) -> e = c*n + i -> block e//4, slot e%4
    for (i, c) in [(0, 0), (1, 0), (2, 0), (3, 0), (36, 4), (10, 2)]:
        e = c * n + i
        b, s = divmod(e, 4)
        ua, ub = (u[b, 0], u[b, 1]) if s < 2 else (u[b, 2], u[b, 3])
        rad = np.sqrt(-2.0 * np.log(ua))
        g = rad * (np.cos(2 * np.pi * ub) if s % 2 == 0 else np.sin(2 * np.pi * ub))
        assert om[i, c] == g


def test_gaussian_distribution():
    om = P.gaussian_matrix(4000, 25, 11).ravel()
    assert abs(om.mean()) < 0.01
    assert abs(om.var() - 1.0) < 0.02
    assert scipy.stats.kstest(om, "norm").pvalue > 1e-3


def test_seeds_differ():
    a = P.gaussian_matrix(100, 3, 1)
    b = P.gaussian_matrix(100, 3, 2)
    assert not np.allclose(a, b)
