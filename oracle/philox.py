"""Philox4x32-10 and the Gaussian blocks Omega drawn by ARA (oracle; test infrastructure).

Algorithm 1 and Algorithm 5 (batchRandn) draw Gaussian sampling blocks Omega of
size b x bs.  The CUDA path draws them on the device; this module is the
oracle's own implementation of the same counter-based generator, written from
its published definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11 (Philox-4x32, 10 rounds,
multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /
0xBB67AE85).

Block layout (a reading of Algorithm 5, shared by both sides by definition):
Omega for (seed, stream, column k, round t) is b x bs, column-major; element
e = c*b + r belongs to pair m = e // 2.  Pair m uses counter
(m, t, k, stream) and key (seed & 0xffffffff, seed >> 32).  The four 32-bit
outputs w0..w3 give u1 = ((w1:w0 as 64 bits) >> 11) + 0.5) * 2^-53 and
u2 = ((w3:w2) >> 11) * 2^-53 + 2^-54; then (Box-Muller)
rho = sqrt(-2 ln u1), z[2m] = rho cos(2 pi u2), z[2m+1] = rho sin(2 pi u2).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Apply Philox4x32 with 10 rounds to counters `ctr` (shape (n, 4), uint32-valued).

    Returns (n, 4) uint64 array holding the 32-bit outputs.
    """
    c = [ctr[:, i].astype(np.uint64) & MASK32 for i in range(4)]
    k0, k1 = key[0] & 0xFFFFFFFF, key[1] & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c[0]  # exact in uint64: 32x32 -> 64 bits
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack(c, axis=1)


def omega(seed: int, stream: int, k: int, t: int, b: int, bs: int) -> np.ndarray:
    """Gaussian block Omega (b x bs, float64) for (seed, stream, column k, round t)."""
    n = b * bs
    m = np.arange((n + 1) // 2, dtype=np.uint64)
    ctr = np.stack([m, np.full_like(m, t), np.full_like(m, k), np.full_like(m, stream)], axis=1)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    a = (w[:, 1] << np.uint64(32)) | w[:, 0]
    c = (w[:, 3] << np.uint64(32)) | w[:, 2]
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = (c >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 + 2.0 ** -54
    rho = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * len(m))
    z[0::2] = rho * np.cos(2.0 * np.pi * u2)
    z[1::2] = rho * np.sin(2.0 * np.pi * u2)
    return z[:n].reshape(bs, b).T.copy()  # column-major element order -> (b, bs)
