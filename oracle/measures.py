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


def backward_error(apply_A, apply_F, x0: np.ndarray, iters: int = 30) -> float:
    """||A - F||_2 / ||A||_2 with F the factored product (L L^T or L D L^T)."""
    nE = power_norm(lambda v: apply_A(v) - apply_F(v), x0, iters)
    nA = power_norm(apply_A, x0, iters)
    return nE / nA


def residual(apply_A, X: np.ndarray, Y: np.ndarray) -> float:
    """||A X - Y||_F / ||Y||_F."""
    return float(np.linalg.norm(apply_A(X) - Y) / np.linalg.norm(Y))
