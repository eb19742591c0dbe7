"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the factorization method: it only draws
points, right-hand sides, power-iteration start vectors and synthetic low-rank
tiles of a prescribed spectrum from fixed seeds.
Random numbers the method itself draws (the ARA Gaussian blocks) are NOT
generated here; each side implements its own counter-based generator.

Generator: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), one 64-bit output per double, top 53 bits scaled to
[0, 1).  The workloads follow the paper's experiments (Section 6): points
uniform in the unit square / cube, an exponential covariance kernel with
length scale 0.1 (2D) or 0.2 (3D) and a small nugget.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)


def _splitmix64(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` consecutive splitmix64 outputs of the stream (seed, stream)."""
    with np.errstate(over="ignore"):
        s0 = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _STREAM_MUL
        n = np.arange(1, count + 1, dtype=np.uint64)
        z = s0 + n * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` doubles uniform in [0, 1) (53-bit resolution)."""
    z = _splitmix64(seed, stream, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` standard normal doubles (Box-Muller on pairs of uniforms)."""
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def points(N: int, d: int, seed: int) -> np.ndarray:
    """N points uniform in [0,1]^d, row-major (N, d) float64, stream 0."""
    return uniform(seed, 0, N * d).reshape(N, d)


def rhs(N: int, nrhs: int, seed: int) -> np.ndarray:
    """N x nrhs standard normal right-hand sides, column-major (Fortran) float64, stream 1."""
    return np.asfortranarray(gaussian(seed, 1, N * nrhs).reshape(nrhs, N).T)


def start_vector(N: int, seed: int = 12345) -> np.ndarray:
    """Gaussian start vector for power iterations (stream 2)."""
    return gaussian(seed, 2, N)


def lowrank_tiles(ntiles: int, b: int, r: int, seed: int, smax: float = 10.0, smin: float = 1e-10):
    """Synthetic low-rank tiles Q_t B_t^T with a prescribed spectrum (rank-trimming inputs): Q_t and W_t
    (b x r) and Z_t (r x r) with orthonormal columns (orthonormalized Gaussians), s_t log-spaced from smax
    down to smin with a seeded jitter of up to a tenth of a step, and B_t = W_t diag(s_t) Z_t^T, so that the
    singular values of Q_t B_t^T are s_t exactly.  Returns Q, B (ntiles, b, r) and s (ntiles, r), stream 3."""
    g = gaussian(seed, 3, ntiles * (2 * b * r + r * r + r))
    Q = np.empty((ntiles, b, r))
    B = np.empty((ntiles, b, r))
    s = np.empty((ntiles, r))
    step = (np.log10(smax) - np.log10(smin)) / max(r - 1, 1)
    o = 0
    for t in range(ntiles):
        Qt = np.linalg.qr(g[o:o + b * r].reshape(b, r))[0]; o += b * r
        Wt = np.linalg.qr(g[o:o + b * r].reshape(b, r))[0]; o += b * r
        Zt = np.linalg.qr(g[o:o + r * r].reshape(r, r))[0]; o += r * r
        jit = 0.1 * step * np.tanh(g[o:o + r]); o += r
        st = 10.0 ** (np.log10(smax) - step * np.arange(r) + jit)
        Q[t], B[t], s[t] = Qt, (Wt * st) @ Zt.T, st
    return Q, B, s


# Workload recipes (paper Section 6 and the covariance configurations used by
# the tests and the bench).  Each entry: N, d, length scale, nugget, tile b,
# ARA block bs, seed.
WORKLOADS = {
    "cov2d_4k": dict(N=4096, d=2, ell=0.1, nugget=1e-4, b=256, bs=16, seed=0),
    "cov3d_32k": dict(N=32768, d=3, ell=0.2, nugget=1e-4, b=512, bs=32, seed=1),
    "cov2d_131k": dict(N=131072, d=2, ell=0.1, nugget=1e-4, b=1024, bs=16, seed=2),
    # smaller case of the same 2D recipe (profiling captures)
    "cov2d_16k": dict(N=16384, d=2, ell=0.1, nugget=1e-4, b=1024, bs=16, seed=2),
}
