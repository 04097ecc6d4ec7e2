"""Gaussian test matrix Omega for the randomized warmstart (oracle).

Algorithm 2 draws Omega ~ N(0,1)^{n x (m0+p)} (also Assumption 1.6). The paper
names no generator, so both this oracle and the CUDA library implement the
same counter-based generator from its published definition:

* Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC'11): 10 rounds of two 64x64->128 multiplies with the
  constants 0xD2E7470EE14C6C93 and 0xCA5A826395121157, key schedule with
  the Weyl increments 0x9E3779B97F4A7C15 and 0xBB67AE8584CAA73B.
* uniform u = ((x >> 11) + 1) * 2^-53 in (0, 1];
* Box-Muller: r = sqrt(-2 ln u0), g0 = r cos(2 pi u1), g1 = r sin(2 pi u1).

Omega is column-major (entry (i, c) has linear index e = c*n + i). Block
b = e // 4 uses counter (b, 0, 0, 0) and key (seed, 0); its four words give
the normals of linear indices 4b..4b+3 as (g0, g1) from words (0, 1) and
(g0, g1) from words (2, 3).

Pinned against ``numpy.random.Philox`` (the same Philox-4x64-10 rounds) in
tests/test_oracle_philox.py.
"""
from __future__ import annotations

import numpy as np

_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B
_MASK = (1 << 64) - 1


def philox4x64_10(ctr, key):
    """One Philox-4x64-10 block for a single counter (python ints)."""
    x0, x1, x2, x3 = (int(v) & _MASK for v in ctr)
    k0, k1 = (int(v) & _MASK for v in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * x0
        p1 = _M1 * x2
        hi0, lo0 = p0 >> 64, p0 & _MASK
        hi1, lo1 = p1 >> 64, p1 & _MASK
        x0, x1, x2, x3 = (hi1 ^ x1 ^ k0), lo1, (hi0 ^ x3 ^ k1), lo0
    return x0, x1, x2, x3


def _mulhilo(a: np.ndarray, m: int):
    """Vectorised 64x64 -> (hi, lo) product on uint64 arrays."""
    a = a.astype(np.uint64)
    m_lo = np.uint64(m & 0xFFFFFFFF)
    m_hi = np.uint64(m >> 32)
    a_lo = a & np.uint64(0xFFFFFFFF)
    a_hi = a >> np.uint64(32)
    ll = a_lo * m_lo
    lh = a_lo * m_hi
    hl = a_hi * m_lo
    hh = a_hi * m_hi
    mid = (ll >> np.uint64(32)) + (lh & np.uint64(0xFFFFFFFF)) + (hl & np.uint64(0xFFFFFFFF))
    lo = (ll & np.uint64(0xFFFFFFFF)) | (mid << np.uint64(32))
    hi = hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))
    return hi, lo


def philox_blocks(counters: np.ndarray, seed: int) -> np.ndarray:
    """Philox-4x64-10 on counters (b, 0, 0, 0) for every b in ``counters``;
    key (seed, 0). Returns uint64 array [len(counters), 4]."""
    with np.errstate(over="ignore"):
        b = np.asarray(counters, dtype=np.uint64)
        x0 = b.copy()
        x1 = np.zeros_like(b)
        x2 = np.zeros_like(b)
        x3 = np.zeros_like(b)
        k0 = np.uint64(seed & _MASK)
        k1 = np.uint64(0)
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint64((int(k0) + _W0) & _MASK)
                k1 = np.uint64((int(k1) + _W1) & _MASK)
            hi0, lo0 = _mulhilo(x0, _M0)
            hi1, lo1 = _mulhilo(x2, _M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=1)


def uniforms(words: np.ndarray) -> np.ndarray:
    """64-bit words -> doubles in (0, 1]."""
    return ((words >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def gaussian_matrix(n: int, k: int, seed: int) -> np.ndarray:
    """Omega in R^{n x k}, entries N(0,1), column-major linear indexing."""
    total = n * k
    nblk = (total + 3) // 4
    words = philox_blocks(np.arange(nblk, dtype=np.uint64), seed)
    u = uniforms(words)
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    g = np.empty((nblk, 4), dtype=np.float64)
    g[:, 0] = r01 * np.cos(2.0 * np.pi * u[:, 1])
    g[:, 1] = r01 * np.sin(2.0 * np.pi * u[:, 1])
    g[:, 2] = r23 * np.cos(2.0 * np.pi * u[:, 3])
    g[:, 3] = r23 * np.sin(2.0 * np.pi * u[:, 3])
    flat = g.ravel()[:total]
    return flat.reshape(k, n).T.copy()


def philox_words(n: int, k: int, seed: int) -> np.ndarray:
    """Raw 64-bit words behind ``gaussian_matrix`` (bit-exact parity)."""
    nblk = (n * k + 3) // 4
    return philox_blocks(np.arange(nblk, dtype=np.uint64), seed)
