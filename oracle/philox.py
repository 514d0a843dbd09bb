"""Philox4x32-10 counter-based generator and the Gaussian start vectors of the
null-vector setup.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The setup ("Setup procedure") starts each null vector from a random vector.
So that the oracle and the CUDA path start from the same vector without
shipping it, both sides implement one counter-based generator from its
published definition: Philox4x32 with 10 rounds (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11).  One round maps counter ``(c0, c1, c2, c3)`` and key ``(k0, k1)`` to
``(hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))`` with
``M0 = 0xD2511F53``, ``M1 = 0xCD9E8D57``; the key is bumped by the Weyl
constants ``(0x9E3779B9, 0xBB67AE85)`` between rounds.

Start vector (a reading; the paper only says "a random vector"): component
``dof`` of site ``lex`` (x fastest) of vector ``k`` on level ``level`` uses
counter ``(lex, dof, k, level)`` and key ``(seed mod 2^32, seed div 2^32)``;
with ``u_i = (w_i + 1/2) 2^-32`` the value is
``sqrt(-ln u_0) * (cos(2 pi u_1) + i sin(2 pi u_1))`` (Box-Muller), so Re and
Im are N(0, 1/2).
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10.  ``ctr``: four uint32 arrays (broadcastable);
    ``key``: two ints.  Returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in ctr)
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def gaussian_vector(seed: int, level: int, k: int, shape, ndof: int) -> np.ndarray:
    """Start vector ``k`` of level ``level`` on a lattice of array shape
    ``(Lt, Lz, Ly, Lx)`` with ``ndof`` components per site."""
    nsite = int(np.prod(shape))
    lex = np.arange(nsite, dtype=np.uint64)[:, None]
    dof = np.arange(ndof, dtype=np.uint64)[None, :]
    w0, w1, _, _ = philox4x32_10((lex, dof, np.uint64(k), np.uint64(level)),
                                 (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    u0 = (w0.astype(np.float64) + 0.5) * 2.0 ** -32
    u1 = (w1.astype(np.float64) + 0.5) * 2.0 ** -32
    rad = np.sqrt(-np.log(u0))
    v = rad * np.cos(2.0 * np.pi * u1) + 1j * rad * np.sin(2.0 * np.pi * u1)
    return v.reshape(tuple(shape) + (ndof,))
