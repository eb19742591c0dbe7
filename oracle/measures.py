"""Accuracy measures (oracle; test infrastructure).

Section 6: "all results were verified by estimating the 2-norm of the
difference ||A - L L^T|| using the power iteration method".  The relative
backward error ||A - L L^T||_2 / ||A||_2 is estimated with a fixed number of
power iterations from a seeded Gaussian start vector (E = A - L L^T is
symmetric, so ||E x|| / ||x|| converges to |lambda_max(E)| = ||E||_2).
"""
from __future__ import annotations

import numpy as np


def power_norm(apply, x0: np.ndarray, iters: int = 30) -> float:
    """Estimate ||M||_2 of a symmetric operator by `iters` power iterations."""
    v = x0 / np.linalg.norm(x0)
    lam = 0.0
    for _ in range(iters):
        w = apply(v)
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


def power_norms(apply_block, X0: np.ndarray, iters: int = 30) -> np.ndarray:
    """Independent power iterations, one per column of X0 (N x m): column c estimates ||M_c||_2 of
    its own symmetric operator.  apply_block(V) returns [M_0 v_0 | ... | M_{m-1} v_{m-1}], so that
    one pass over an expensive shared operand (the exact kernel matrix) serves every column.
    Each column follows power_norm's steps: w = M v, lam = ||w||, v = w / lam (0 stays 0)."""
    V = np.array(X0, dtype=np.float64, copy=True).reshape(X0.shape[0], -1)
    V /= np.linalg.norm(V, axis=0)
    m = V.shape[1]
    lam = np.zeros(m)
    live = np.ones(m, dtype=bool)
    for _ in range(iters):
        W = apply_block(V)
        for c in range(m):
            if not live[c]:
                continue
            lam[c] = float(np.linalg.norm(W[:, c]))
            if lam[c] == 0.0:
                live[c] = False
            else:
                V[:, c] = W[:, c] / lam[c]
    return lam


def backward_error(apply_A, apply_F, x0: np.ndarray, iters: int = 30) -> float:
    """||A - F||_2 / ||A||_2 with F the factored product (L L^T or L D L^T)."""
    nE = power_norm(lambda v: apply_A(v) - apply_F(v), x0, iters)
    nA = power_norm(apply_A, x0, iters)
    return nE / nA


def residual(apply_A, X: np.ndarray, Y: np.ndarray) -> float:
    """||A X - Y||_F / ||Y||_F."""
    return float(np.linalg.norm(apply_A(X) - Y) / np.linalg.norm(Y))
