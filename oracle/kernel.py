"""Exponential covariance kernel tiles (oracle; test infrastructure).

Section 6: covariance matrices of spatial Gaussian processes with an isotropic
exponential kernel, A_ij = exp(-||x_i - x_j||_2 / ell), plus a nugget on the
diagonal (A_ii = 1 + nugget).  Rows/columns past N (the padding of a ragged
last tile, Section 6 clustering paragraph) are identity rows/columns.
"""
from __future__ import annotations

import numpy as np


def kernel_block(xr: np.ndarray, xc: np.ndarray, ell: float) -> np.ndarray:
    """exp(-||xr_i - xc_j|| / ell) for all pairs (no nugget)."""
    diff = xr[:, None, :] - xc[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    return np.exp(-r / ell)


def tile(xo: np.ndarray, i: int, j: int, b: int, ell: float, nugget: float) -> np.ndarray:
    """Dense b x b tile (i, j) of the kernel matrix of the ordered points `xo`, identity-padded."""
    N = xo.shape[0]
    T = np.zeros((b, b))
    r0, c0 = i * b, j * b
    r1, c1 = min(r0 + b, N), min(c0 + b, N)
    if r1 > r0 and c1 > c0:
        T[: r1 - r0, : c1 - c0] = kernel_block(xo[r0:r1], xo[c0:c1], ell)
    if i == j:
        n = max(r1 - r0, 0)
        T[np.arange(n), np.arange(n)] += nugget
        T[np.arange(n, b), np.arange(n, b)] = 1.0  # padding
    return T


def dense(xo: np.ndarray, ell: float, nugget: float) -> np.ndarray:
    """Full N x N kernel matrix (small N only)."""
    A = kernel_block(xo, xo, ell)
    A[np.diag_indices_from(A)] += nugget
    return A


def matvec(xo: np.ndarray, ell: float, nugget: float, X: np.ndarray, chunk: int = 2048) -> np.ndarray:
    """A @ X with A generated on the fly in row chunks (exact kernel matrix)."""
    N = xo.shape[0]
    X = X.reshape(N, -1)
    Y = np.empty_like(X)
    for r0 in range(0, N, chunk):
        r1 = min(r0 + chunk, N)
        Y[r0:r1] = kernel_block(xo[r0:r1], xo, ell) @ X
    Y += nugget * X
    return Y
