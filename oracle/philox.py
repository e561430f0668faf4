"""Philox-4x32-10 and the Gaussian test matrices of Algorithm 1 (oracle side).

Algorithm 1 draws a fresh Omega in C^{K x d} with i.i.d. CN(0,1) entries in every iteration.
Both this oracle and the CUDA path draw Omega from the same counter-based generator, each
with its own implementation written from the published definition:

  J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as
  1, 2, 3", SC'11 -- the Philox-4x32 bijection with multipliers 0xD2511F53 / 0xCD9E8D57,
  Weyl key increments 0x9E3779B9 / 0xBB67AE85, 10 rounds.

Counter layout (shared convention, not shared code): entry Omega[i, j] of iteration `it`
at update step `t` of instance `b` uses counter (c0, c1, c2, c3) = (i, j // 2, t, 16 b + it)
and key (seed mod 2^32, seed >> 32).  The four output words (x0, x1, x2, x3) give entry
j = 2q from (x0, x1) and entry j = 2q + 1 from (x2, x3).

Uniforms: u(x) = ((x >> 9) + 0.5) * 2^-23, exactly representable in binary32 and binary64
and strictly inside (0, 1).  Box-Muller for a circular complex Gaussian of unit variance:
omega = sqrt(-ln u(x_a)) * exp(j 2 pi u(x_b)); |omega|^2 = -ln u is Exp(1) and the phase is
uniform, so Re and Im are independent N(0, 1/2).
"""
from __future__ import annotations

import numpy as np

_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF


def _mulhilo(a: np.ndarray, b: int) -> tuple[np.ndarray, np.ndarray]:
    prod = a.astype(np.uint64) * np.uint64(b)
    return (prod >> np.uint64(32)).astype(np.uint64), (prod & np.uint64(_MASK)).astype(np.uint64)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox-4x32 with 10 rounds.

    ctr: array-like [..., 4] of uint32 counters; key: array-like [..., 2] of uint32 keys
    (broadcast against ctr).  Returns uint32 [..., 4].
    """
    c = np.asarray(ctr, dtype=np.uint64) & np.uint64(_MASK)
    k = np.broadcast_to(np.asarray(key, dtype=np.uint64) & np.uint64(_MASK),
                        c.shape[:-1] + (2,))
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for rnd in range(10):
        if rnd > 0:  # key schedule: bump before every round but the first
            k0 = (k0 + np.uint64(_W0)) & np.uint64(_MASK)
            k1 = (k1 + np.uint64(_W1)) & np.uint64(_MASK)
        hi0, lo0 = _mulhilo(c0, _M0)
        hi1, lo1 = _mulhilo(c2, _M1)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniform_open01(x: np.ndarray) -> np.ndarray:
    """Map uint32 words to (0, 1): ((x >> 9) + 0.5) * 2^-23 in float64."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(xa: np.ndarray, xb: np.ndarray) -> np.ndarray:
    """CN(0,1) sample from two uint32 words: sqrt(-ln u_a) * exp(j 2 pi u_b)."""
    ua = uniform_open01(xa)
    ub = uniform_open01(xb)
    rad = np.sqrt(-np.log(ua))
    ang = 2.0 * np.pi * ub
    return rad * np.cos(ang) + 1j * rad * np.sin(ang)


def omega(K: int, d: int, *, seed: int, step: int, instance: int, it: int) -> np.ndarray:
    """Algorithm 1's test matrix Omega in C^{K x d} for one (instance, step, iteration)."""
    assert 0 <= it < 16 and K >= 1 and d >= 1
    nq = (d + 1) // 2
    i_idx, q_idx = np.meshgrid(np.arange(K), np.arange(nq), indexing="ij")
    ctr = np.stack([i_idx, q_idx,
                    np.full_like(i_idx, step & _MASK),
                    np.full_like(i_idx, (16 * instance + it) & _MASK)], axis=-1)
    key = np.array([seed & _MASK, (seed >> 32) & _MASK], dtype=np.uint64)
    x = philox4x32_10(ctr, key)                          # [K, nq, 4]
    even = box_muller(x[..., 0], x[..., 1])              # columns 2q
    odd = box_muller(x[..., 2], x[..., 3])               # columns 2q + 1
    out = np.empty((K, 2 * nq), dtype=np.complex128)
    out[:, 0::2] = even
    out[:, 1::2] = odd
    return out[:, :d]
