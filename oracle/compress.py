"""Tile compressors (oracle; test infrastructure).

svd_truncate: the reference compressor prescribed for the oracle: keep the
  smallest rank r with sigma_{r+1} <= eps (an absolute 2-norm threshold, as
  Section 6 states), so ||T - Q B^T||_2 <= eps
  (Eckart-Young).  Q = U_r (orthonormal), B = V_r Sigma_r.

trim: ARA -> SVD rank trimming of a compressed tile (Q B^T -> its truncated
  SVD, through the SVD of the short factor B).

ara: Adaptive Randomized Approximation, Algorithm 1 (Section 3.1), applied to
  a dense operand T.  Steps in the paper's order: draw Omega (b x bs), sample
  Y = T Omega, orthog(Q, Y) = two iterations of block Gram-Schmidt against Q,
  each followed by a Cholesky-QR of the panel, append, convergence test; at
  the end project B = T^T Q (Algorithm 5, sampleLeftT).

  Readings (the paper defers the details of orthog/convergence to its ref.
  on batched ARA, which is not reproduced in the paper):
  * convergence(R): e = max over the bs new columns of ||(I - Q Q^T) T w_c||_2,
    taken from the first Gram-Schmidt iteration (the column norms of the
    projected panel, i.e. the column norms of its R factor).  The loop stops
    when e <= eps / (10 sqrt(2/pi)) -- the a-posteriori bound of Halko,
    Martinsson, Tropp (2011, Lemma 4.1 / Alg. 4.2) that then gives
    ||T - Q Q^T T||_2 <= eps with probability >= 1 - 10^-bs.  A block that
    passes the test only certifies the basis: it is not appended (appending it
    would raise every rank by bs, while the paper reports ARA ranks within a
    few percent of SVD ranks, Section 6.2).
  * Cholesky-QR of the first iteration drops a panel column whose pivot (its
    squared norm orthogonal to Q and to the kept earlier columns) is below
    max(thr^2, tau * G_jj), tau = 1e-10: such a direction carries less than
    the threshold, or cannot be resolved through the Gram matrix; the
    a-posteriori test of the next round re-detects anything that matters.
  * the rank is capped at min(m, n) of T.
"""
from __future__ import annotations

import math

import numpy as np

TAU_DROP = 1e-10
HALKO = 10.0 * math.sqrt(2.0 / math.pi)


def svd_truncate(T: np.ndarray, eps: float) -> tuple[np.ndarray, np.ndarray]:
    """T ~= Q B^T with the smallest rank r such that sigma_{r+1} <= eps."""
    U, s, Vt = np.linalg.svd(T, full_matrices=False)
    r = int(np.count_nonzero(s > eps))
    return U[:, :r].copy(), (Vt[:r].T * s[:r]).copy()


def trim(Q: np.ndarray, B: np.ndarray, eps: float) -> tuple[np.ndarray, np.ndarray]:
    """ARA -> SVD rank trimming of a tile Q B^T with orthonormal Q (b x r): the SVD of the short factor,
    B = W S Z^T, gives Q B^T = (Q Z) S W^T, whose singular values are S; keep those above eps.
    Returns (Q Z_r, W_r S_r): the rank the truncated SVD of the tile would keep, error <= eps."""
    if B.shape[1] == 0:
        return Q.copy(), B.copy()
    W, sv, Zt = np.linalg.svd(B, full_matrices=False)
    r = int(np.count_nonzero(sv > eps))
    return Q @ Zt[:r].T, W[:, :r] * sv[:r]


def chol_drop(G: np.ndarray, thr2: float, tau: float = TAU_DROP) -> tuple[np.ndarray, list[int]]:
    """Unpivoted Cholesky G = R^T R restricted to the columns it keeps.

    Column j is processed in order; its pivot d = G_jj - sum_{l kept} R_lj^2 is the
    squared norm of column j orthogonal to the kept earlier columns.  It is dropped
    when d <= max(thr2, tau * G_jj).  Returns (R restricted to kept rows/cols, kept).
    """
    n = G.shape[0]
    R = np.zeros((n, n))
    keep: list[int] = []
    for j in range(n):
        for p, l in enumerate(keep):
            prev = keep[:p]
            R[l, j] = (G[l, j] - R[prev, l] @ R[prev, j]) / R[l, l]
        d = G[j, j] - sum(R[l, j] ** 2 for l in keep)
        if d <= max(thr2, tau * G[j, j]) or not d > 0.0:
            continue
        R[j, j] = math.sqrt(d)
        keep.append(j)
    return R[np.ix_(keep, keep)], keep


def orthog(Q: np.ndarray, Y: np.ndarray, thr: float) -> tuple[np.ndarray | None, float]:
    """orthog(Q, Y) of Algorithm 1 with its convergence quantity.

    Returns (Z, e): Z = orthonormal columns to append (None if converged), e = max
    column norm of (I - Q Q^T) Y.
    """
    # block Gram-Schmidt, iteration 1
    Y1 = Y - Q @ (Q.T @ Y)
    G1 = Y1.T @ Y1
    e = math.sqrt(max(float(np.max(np.diag(G1))), 0.0)) if G1.size else 0.0
    if e <= thr:
        return None, e
    R1, keep = chol_drop(G1, thr * thr)
    W = np.linalg.solve(R1.T, Y1[:, keep].T).T  # W R1 = Y1[:, keep]
    # block Gram-Schmidt, iteration 2 (re-orthogonalization)
    Y2 = W - Q @ (Q.T @ W)
    G2 = Y2.T @ Y2
    R2, keep2 = chol_drop(G2, 0.0)
    Z = np.linalg.solve(R2.T, Y2[:, keep2].T).T
    return Z, e


def ara(apply_T, m: int, n: int, bs: int, eps: float, omega_of_round, apply_Tt=None,
        max_rank: int | None = None) -> tuple[np.ndarray, np.ndarray, int]:
    """Algorithm 1 on the m x n operator T given as callables.

    apply_T(Omega) = T @ Omega (Omega: n x bs); apply_Tt(Q) = T^T @ Q.
    omega_of_round(t) -> n x bs Gaussian block for round t (t = 0, 1, ...).
    Returns (Q, B, rounds) with T ~= Q B^T.
    """
    cap = min(m, n) if max_rank is None else max_rank
    thr = eps / HALKO
    Q = np.zeros((m, 0))
    t = 0
    while Q.shape[1] < cap:
        Om = omega_of_round(t)
        t += 1
        Y = apply_T(Om)
        Z, e = orthog(Q, Y, thr)
        if Z is None:
            break
        Q = np.hstack([Q, Z[:, : cap - Q.shape[1]]])
    B = apply_Tt(Q) if apply_Tt is not None else None
    return Q, B, t


def ara_dense(T: np.ndarray, bs: int, eps: float, omega_of_round) -> tuple[np.ndarray, np.ndarray, int]:
    """ARA of a dense tile: T ~= Q B^T."""
    return ara(lambda Om: T @ Om, T.shape[0], T.shape[1], bs, eps, omega_of_round,
               apply_Tt=lambda Q: T.T @ Q)
