"""Dense factorizations and triangular solves (oracle; test infrastructure).

Section 3.2: dense Cholesky A = L L^T (column by column: the diagonal entry is
the square root of the updated pivot, the column below is scaled by it).
Section 5.3 / Algorithm 10: unpivoted LDL^T of a diagonal tile,
A = L D L^T with L unit lower triangular and D diagonal (1x1 pivots, no
pivoting, as the factorization is pivot-free).

Written as textbook column loops (left-looking, one column at a time) so that
each line can be checked by eye; numpy provides the vector operations.
"""
from __future__ import annotations

import numpy as np


class NotPositiveDefinite(Exception):
    """A pivot was not positive (Cholesky) or was zero (LDL^T); `.index` is its column."""

    def __init__(self, index: int):
        super().__init__(f"non-positive pivot at column {index}")
        self.index = index


def cholesky(A: np.ndarray) -> np.ndarray:
    """Lower-triangular L with A = L L^T (reads the lower triangle of A)."""
    n = A.shape[0]
    L = np.zeros_like(A, dtype=np.float64)
    for j in range(n):
        # pivot: a_jj - sum_{k<j} l_jk^2
        d = A[j, j] - L[j, :j] @ L[j, :j]
        if not d > 0.0:
            raise NotPositiveDefinite(j)
        L[j, j] = np.sqrt(d)
        # column below: (a_ij - sum_{k<j} l_ik l_jk) / l_jj
        L[j + 1 :, j] = (A[j + 1 :, j] - L[j + 1 :, :j] @ L[j, :j]) / L[j, j]
    return L


def ldlt(A: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Unit lower L and diagonal d with A = L diag(d) L^T, no pivoting."""
    n = A.shape[0]
    L = np.eye(n)
    d = np.zeros(n)
    for j in range(n):
        # d_j = a_jj - sum_{k<j} l_jk^2 d_k
        d[j] = A[j, j] - (L[j, :j] * d[:j]) @ L[j, :j]
        if d[j] == 0.0:
            raise NotPositiveDefinite(j)
        # l_ij = (a_ij - sum_{k<j} l_ik d_k l_jk) / d_j
        L[j + 1 :, j] = (A[j + 1 :, j] - L[j + 1 :, :j] @ (d[:j] * L[j, :j])) / d[j]
    return L, d


def solve_lower(L: np.ndarray, B: np.ndarray, unit: bool = False) -> np.ndarray:
    """X with L X = B (forward substitution, row by row)."""
    B = np.array(B, dtype=np.float64, copy=True)
    vec = B.ndim == 1
    X = B.reshape(B.shape[0], -1)
    n = L.shape[0]
    for i in range(n):
        X[i] -= L[i, :i] @ X[:i]
        if not unit:
            X[i] /= L[i, i]
    return X[:, 0] if vec else X


def solve_upper_t(L: np.ndarray, B: np.ndarray, unit: bool = False) -> np.ndarray:
    """X with L^T X = B (backward substitution with the transpose of lower L)."""
    B = np.array(B, dtype=np.float64, copy=True)
    vec = B.ndim == 1
    X = B.reshape(B.shape[0], -1)
    n = L.shape[0]
    for i in range(n - 1, -1, -1):
        X[i] -= L[i + 1 :, i] @ X[i + 1 :]
        if not unit:
            X[i] /= L[i, i]
    return X[:, 0] if vec else X


def _modify_eigenvalues(w: np.ndarray, delta: float) -> np.ndarray:
    """modifySPD (Algorithm 8) on one pivot block's eigenvalues: those below delta are raised to it."""
    return np.maximum(w, delta)


def modified_cholesky(A: np.ndarray, delta: float | None = None):
    """ModChol (Algorithm 8, Section 5.1.2): the Cholesky factor of A if A is positive definite
    (E = 0); otherwise the factor of A + E from a symmetric indefinite factorization
    A = Lp D Lp^T (Bunch-Kaufman pivoting, SciPy's ldl as one step; Lp is a row-permuted unit lower
    triangle) whose 1x1 and 2x2 diagonal blocks are modified as in Cheng and Higham (1998): each
    block's eigenvalues are raised to at least delta (default sqrt(u) ||A||_inf, their choice),
    giving D + F positive definite and A + E = Lp (D + F) Lp^T.  Returns (L, ||E||_2)."""
    try:
        return cholesky(A), 0.0
    except NotPositiveDefinite:
        pass
    import scipy.linalg as sl
    n = A.shape[0]
    if delta is None:
        delta = np.sqrt(np.finfo(np.float64).eps / 2) * np.abs(A).sum(axis=1).max()
    Lp, D, _ = sl.ldl(A, lower=True)
    DF = np.zeros_like(D)
    i = 0
    while i < n:
        if i + 1 < n and D[i + 1, i] != 0.0:  # a 2 x 2 block
            w, Q = np.linalg.eigh(D[i:i + 2, i:i + 2])
            DF[i:i + 2, i:i + 2] = (Q * _modify_eigenvalues(w, delta)) @ Q.T
            i += 2
        else:
            DF[i, i] = _modify_eigenvalues(np.array([D[i, i]]), delta)[0]
            i += 1
    At = Lp @ DF @ Lp.T
    At = 0.5 * (At + At.T)
    return cholesky(At), float(np.linalg.norm(At - A, 2))
