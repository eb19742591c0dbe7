"""Tile low rank matrix, left-looking TLR Cholesky / LDL^T, solve, logdet (oracle; test infrastructure).

Format (Section 1, Figure 1): the N x N matrix (points in KD order, padded to
nb*b with identity rows) is cut into b x b tiles; diagonal tiles are dense,
each lower off-diagonal tile (i, j), i > j, is U_ij V_ij^T.

Factorization: Algorithm 6 (Cholesky) / Algorithm 10 (LDL^T), left looking.
For k = 0 .. nb-1:
  * updateDense (Section 4.3): D_k = sum_{j<k} L(k,j) L(k,j)^T
      = sum_j U_kj (V_kj^T V_kj) U_kj^T   (LDL^T: V_kj^T D_j V_kj in the middle),
    A(k,k) <- A(k,k) - D_k (+ compensation, Section 5.1);
  * chol / ldl of the diagonal tile;
  * every tile below: T = A(i,k) - sum_{j<k} U_ij V_ij^T [D_j] V_kj U_kj^T
    (Equation 1 / Equation 3), formed densely here, compressed to eps
    (truncated SVD by default, or ARA with the same Gaussian blocks as the
    CUDA path), T ~= Q B^T;
  * batchTrsm: V_ik = L_kk^{-1} B (LDL^T: D_k^{-1} L_kk^{-1} B, batchIDMult),
    U_ik = Q (Section 4.3: compress first, then the triangular solve).
Solve: Algorithm 7 (forward), its transpose (backward), D^{-1} in between for LDL^T.
logdet: 2 sum log diag(L_kk) (Cholesky) or sum log|D| (LDL^T).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import compress as C
from . import dense as Dn
from . import kdtree, kernel, philox

STREAM_COMPRESS = 1
STREAM_FACTOR = 2
STREAM_SCHUR = 3


@dataclass
class TLR:
    N: int
    b: int
    nb: int
    perm: np.ndarray
    xo: np.ndarray
    diag: list = field(default_factory=list)   # dense b x b tiles (A_kk, then L_kk)
    U: dict = field(default_factory=dict)      # (i, j) -> b x r
    V: dict = field(default_factory=dict)
    d: list | None = None                      # LDL^T: D_k as vectors
    kind: str = "A"                            # "A", "chol" or "ldlt"
    rounds: dict = field(default_factory=dict)  # ARA rounds per tile (diagnostics)
    tile_perm: list | None = None              # pivoted factor: original tile at each position

    def rank(self, i: int, j: int) -> int:
        return self.U[(i, j)].shape[1]

    def ranks(self) -> np.ndarray:
        R = np.zeros((self.nb, self.nb), dtype=np.int64)
        for (i, j), u in self.U.items():
            R[i, j] = u.shape[1]
        return R

    def tile_dense(self, i: int, j: int) -> np.ndarray:
        if i == j:
            return self.diag[i]
        if i > j:
            return self.U[(i, j)] @ self.V[(i, j)].T
        return (self.U[(j, i)] @ self.V[(j, i)].T).T

    def to_dense(self) -> np.ndarray:
        """Dense padded matrix (A) or dense L (factors), permuted order."""
        n = self.nb * self.b
        M = np.zeros((n, n))
        b = self.b
        for i in range(self.nb):
            for j in range(self.nb):
                if self.kind != "A" and j > i:
                    continue
                M[i * b:(i + 1) * b, j * b:(j + 1) * b] = self.tile_dense(i, j)
        return M


def _compressor(name: str, eps: float, bs: int, seed: int, stream: int, k: int, b: int):
    if name == "svd":
        return lambda T: (*C.svd_truncate(T, eps), 0)
    if name == "ara":
        return lambda T: C.ara_dense(T, bs, eps, lambda t: philox.omega(seed, stream, k, t, b, bs))
    raise ValueError(name)


def build(points: np.ndarray, b: int, eps: float, ell: float, nugget: float,
          compressor: str = "svd", bs: int = 16, seed: int = 0, mapper=map) -> TLR:
    """KD-order the points and compress every lower off-diagonal tile to eps (Section 6).

    mapper: how the independent tiles of one block column are visited (the builtin map, or the
    map of a thread pool for large cases); every tile is computed the same way either way."""
    points = np.asarray(points, dtype=np.float64)
    N = points.shape[0]
    perm = kdtree.kd_order(points, b)
    xo = points[perm]
    nb = max(1, -(-N // b))
    A = TLR(N=N, b=b, nb=nb, perm=perm, xo=xo)
    A.diag = list(mapper(lambda k: kernel.tile(xo, k, k, b, ell, nugget), range(nb)))
    comp = _compressor(compressor, eps, bs, seed, STREAM_COMPRESS, 0, b)
    for j in range(nb):
        rows = range(j + 1, nb)
        for i, (Q, B, t) in zip(rows, mapper(lambda i: comp(kernel.tile(xo, i, j, b, ell, nugget)), rows)):
            A.U[(i, j)], A.V[(i, j)] = Q, B
            A.rounds[(i, j)] = t
    return A


def _dv(F: TLR, j: int, V: np.ndarray) -> np.ndarray:
    """[D_j] V: V itself for a Cholesky factor, D_j V for LDL^T (Equation 3)."""
    return V if F.d is None else F.d[j][:, None] * V


def _update_sum(F: TLR, i: int, l: int, k: int) -> np.ndarray:
    """sum_{j<k} L(i,j) [D_j] L(l,j)^T = sum_j U_ij (V_ij^T [D_j] V_lj) U_lj^T, formed densely.

    The sum over j is evaluated as one product of the concatenated factors,
    [U_i0 M_0 | ... | U_i,k-1 M_k-1] [U_l0 | ... | U_l,k-1]^T with M_j = V_ij^T [D_j] V_lj:
    the same sum written as a block inner product."""
    b = F.b
    if k == 0:
        return np.zeros((b, b))
    left = np.hstack([F.U[(i, j)] @ (F.V[(i, j)].T @ _dv(F, j, F.V[(l, j)])) for j in range(k)])
    right = np.hstack([F.U[(l, j)] for j in range(k)])
    return left @ right.T


def _diag_update(F: TLR, k: int) -> np.ndarray:
    """D_k = sum_{j<k} L(k,j) [D_j] L(k,j)^T, formed densely (updateDense, Section 4.3)."""
    return _update_sum(F, k, k, k)


def _update_tile(A: TLR, F: TLR, i: int, k: int) -> np.ndarray:
    """Equation 1 / 3, formed densely: T = A(i,k) - sum_{j<k} U_ij V_ij^T [D_j] V_kj U_kj^T."""
    return A.U[(i, k)] @ A.V[(i, k)].T - _update_sum(F, i, k, k)


def _schur_compensation(Dk: np.ndarray, comp) -> np.ndarray:
    """Section 5.1.1: the term added to A(k,k) - D_k, diag(rowsum|D_k - Dbar_k|), with Dbar_k =
    Q Q^T D_k Q Q^T and Q the compressor's eps-basis of the symmetric D_k."""
    Q, _, _ = comp(Dk)
    Dbar = Q @ (Q.T @ Dk @ Q) @ Q.T
    return np.diag(np.sum(np.abs(Dk - Dbar), axis=1))


def factor(A: TLR, eps: float, ldl: bool = False, compressor: str = "svd", bs: int = 16,
           seed: int = 0, compensation: str | None = None, shift: float = 0.0, mapper=map) -> TLR:
    """Left-looking TLR Cholesky (Algorithm 6) or LDL^T (Algorithm 10); returns the factor.

    compensation: None, "shift" (A + shift*I, Section 5.1), "schur"
    (A(k,k) - D_k + diag(rowsum|D_k - Dbar_k|), Section 5.1.1, with Dbar_k the
    compressor's eps-approximation Q Q^T D_k Q Q^T) or "modchol" (Cholesky only:
    a diagonal tile that is not positive definite is factored by the modified
    Cholesky of Algorithm 8, Section 5.1.2).
    mapper: how the independent tiles below the diagonal of one column are visited (builtin map or
    a thread pool's map); each tile's arithmetic is the same either way.
    Raises dense.NotPositiveDefinite with attribute `.tile` on breakdown.
    """
    b, nb = A.b, A.nb
    F = TLR(N=A.N, b=b, nb=nb, perm=A.perm, xo=A.xo, kind="ldlt" if ldl else "chol")
    F.d = [None] * nb if ldl else None
    for k in range(nb):
        Dk = _diag_update(F, k)
        Akk = A.diag[k] - Dk
        if compensation == "shift":
            Akk = Akk + shift * np.eye(b)
        elif compensation == "schur" and k > 0:
            Akk = Akk + _schur_compensation(Dk, _compressor(compressor, eps, bs, seed, STREAM_SCHUR, k, b))
        try:
            if ldl:
                Lkk, dk = Dn.ldlt(Akk)
                F.d[k] = dk
            elif compensation == "modchol":
                Lkk, _ = Dn.modified_cholesky(Akk)   # Algorithm 8 in place of the dense Cholesky
            else:
                Lkk = Dn.cholesky(Akk)
        except Dn.NotPositiveDefinite as ex:
            ex.tile = k
            raise
        F.diag.append(Lkk)
        comp = _compressor(compressor, eps, bs, seed, STREAM_FACTOR, k, b)

        def column_tile(i):
            Q, B, t = comp(_update_tile(A, F, i, k))          # Equation 1 / 3, compressed
            Vik = Dn.solve_lower(Lkk, B, unit=ldl)           # batchTrsm
            if ldl:
                Vik = Vik / F.d[k][:, None]                  # batchIDMult
            return Q, Vik.reshape(b, -1), t

        rows = range(k + 1, nb)
        for i, (Q, Vik, t) in zip(rows, mapper(column_tile, rows)):
            F.U[(i, k)], F.V[(i, k)] = Q, Vik
            F.rounds[(i, k)] = t
    return F


def _row_update(F: TLR, i: int, k: int) -> np.ndarray:
    """D_i = sum_{j<k} L(i,j) L(i,j)^T for a row i >= k of a Cholesky factor in progress (Algorithm 9
    keeps these sums for every remaining diagonal tile, denseUpdates)."""
    return _update_sum(F, i, i, k)


def _select_pivot(Ad: list, D: dict, k: int) -> int:
    """selectPivot (Algorithm 9, Section 5.2): the remaining diagonal tile whose updated value
    A(i,i) - D_i has the largest Frobenius norm; the first such tile on ties."""
    nrm = [np.linalg.norm(Ad[i] - D[i]) for i in range(k, len(Ad))]
    return k + int(np.argmax(nrm))


def _swap_tiles(F: TLR, Ad: list, At: dict, k: int, p: int) -> dict:
    """pivotRowColumn (Algorithm 9): exchange tile rows and columns k and p (k < p) of the symmetric
    trailing matrix and rows k and p of the factored columns.  At holds the trailing lower tiles
    (i, j), i > j >= k, as (U, V) with A(i,j) = U V^T; a tile that crosses to the upper triangle is
    stored transposed (U and V exchanged)."""
    sig = lambda i: p if i == k else (k if i == p else i)
    Ad[k], Ad[p] = Ad[p], Ad[k]
    for j in range(k):
        F.U[(k, j)], F.U[(p, j)] = F.U[(p, j)], F.U[(k, j)]
        F.V[(k, j)], F.V[(p, j)] = F.V[(p, j)], F.V[(k, j)]
    new = {}
    for (i, j) in At:
        a, c = sig(i), sig(j)
        U, V = At[(a, c)] if a > c else At[(c, a)][::-1]
        new[(i, j)] = (U, V)
    return new


def factor_pivoted(A: TLR, eps: float, compressor: str = "svd", bs: int = 16, seed: int = 0) -> TLR:
    """Pivoted left-looking TLR Cholesky (Algorithm 9, Section 5.2): at step k every remaining diagonal
    tile's update D_i is formed, the tile with the largest ||A(i,i) - D_i||_F becomes the pivot, tile
    rows and columns k and pivot are exchanged, and the step continues as in Algorithm 6.  Returns the
    factor of P A P^T; F.perm (point order) includes the tile exchanges and F.tile_perm[k] is the
    original tile at position k, so solves and products in the original order apply A^{-1} and A.
    Requires N to be a multiple of b (no padded tile to move)."""
    b, nb = A.b, A.nb
    assert A.N == nb * b, "pivoted factorization needs N divisible by b"
    F = TLR(N=A.N, b=b, nb=nb, perm=A.perm.copy(), xo=A.xo, kind="chol")
    Ad = [t.copy() for t in A.diag]
    At = {(i, j): (A.U[(i, j)], A.V[(i, j)]) for (i, j) in A.U}
    tp = list(range(nb))
    for k in range(nb):
        D = {i: _row_update(F, i, k) for i in range(k, nb)}
        p = _select_pivot(Ad, D, k)
        if p != k:
            At = _swap_tiles(F, Ad, At, k, p)
            D[k], D[p] = D[p], D[k]
            tp[k], tp[p] = tp[p], tp[k]
        try:
            Lkk = Dn.cholesky(Ad[k] - D[k])
        except Dn.NotPositiveDefinite as ex:
            ex.tile = k
            raise
        F.diag.append(Lkk)
        comp = _compressor(compressor, eps, bs, seed, STREAM_FACTOR, k, b)
        for i in range(k + 1, nb):
            U0, V0 = At[(i, k)]
            Q, B, t = comp(U0 @ V0.T - _update_sum(F, i, k, k))
            F.U[(i, k)], F.V[(i, k)] = Q, Dn.solve_lower(Lkk, B)
            F.rounds[(i, k)] = t
        At = {key: v for key, v in At.items() if key[1] > k}
    F.tile_perm = tp
    F.perm = np.concatenate([A.perm[t * b:(t + 1) * b] for t in tp])
    return F


def _to_perm(F: TLR, Y: np.ndarray) -> np.ndarray:
    Y = np.asarray(Y, dtype=np.float64).reshape(F.N, -1)
    X = np.zeros((F.nb * F.b, Y.shape[1]))
    X[: F.N] = Y[F.perm]
    return X


def _from_perm(F: TLR, X: np.ndarray) -> np.ndarray:
    Y = np.empty((F.N, X.shape[1]))
    Y[F.perm] = X[: F.N]
    return Y


def solve(F: TLR, Y: np.ndarray) -> np.ndarray:
    """X = (L L^T)^{-1} Y or (L D L^T)^{-1} Y; Y in the original point order (N x nrhs)."""
    b, nb = F.b, F.nb
    unit = F.kind == "ldlt"
    X = _to_perm(F, Y)
    blk = lambda k: slice(k * b, (k + 1) * b)
    # forward, Algorithm 7: x(k) = L_kk^{-1} x(k); x(i) -= U_ik (V_ik^T x(k)), i > k
    for k in range(nb):
        X[blk(k)] = Dn.solve_lower(F.diag[k], X[blk(k)], unit=unit)
        for i in range(k + 1, nb):
            X[blk(i)] -= F.U[(i, k)] @ (F.V[(i, k)].T @ X[blk(k)])
    if unit:
        X /= np.concatenate(F.d)[:, None]
    # backward (transpose of Algorithm 7): x(k) -= sum_{i>k} V_ik (U_ik^T x(i)); x(k) = L_kk^{-T} x(k)
    for k in range(nb - 1, -1, -1):
        for i in range(k + 1, nb):
            X[blk(k)] -= F.V[(i, k)] @ (F.U[(i, k)].T @ X[blk(i)])
        X[blk(k)] = Dn.solve_upper_t(F.diag[k], X[blk(k)], unit=unit)
    return _from_perm(F, X)


def logdet(F: TLR) -> float:
    """log det of the factored matrix: 2 sum log diag(L_kk), or sum log|D| for LDL^T."""
    if F.kind == "ldlt":
        return float(sum(np.sum(np.log(np.abs(dk))) for dk in F.d))
    return float(2.0 * sum(np.sum(np.log(np.diag(L))) for L in F.diag))


def matvec(F: TLR, X: np.ndarray, op: str = "LLt") -> np.ndarray:
    """TLR products in the original point order.

    op: "A" (F must be a TLR of A, symmetric product), "L", "Lt", or "LLt"
    (L L^T, or L D L^T for an LDL^T factor).
    """
    b, nb = F.b, F.nb
    Xp = _to_perm(F, X)
    blk = lambda k: slice(k * b, (k + 1) * b)

    def mulL(Z):
        Y = np.zeros_like(Z)
        for i in range(nb):
            Y[blk(i)] = F.diag[i] @ Z[blk(i)]
            for j in range(i):
                Y[blk(i)] += F.U[(i, j)] @ (F.V[(i, j)].T @ Z[blk(j)])
        return Y

    def mulLt(Z):
        Y = np.zeros_like(Z)
        for j in range(nb):
            Y[blk(j)] = F.diag[j].T @ Z[blk(j)]
            for i in range(j + 1, nb):
                Y[blk(j)] += F.V[(i, j)] @ (F.U[(i, j)].T @ Z[blk(i)])
        return Y

    if op == "A":
        Y = np.zeros_like(Xp)
        for i in range(nb):
            Y[blk(i)] += F.diag[i] @ Xp[blk(i)]
            for j in range(i):
                Y[blk(i)] += F.U[(i, j)] @ (F.V[(i, j)].T @ Xp[blk(j)])
                Y[blk(j)] += F.V[(i, j)] @ (F.U[(i, j)].T @ Xp[blk(i)])
    elif op == "L":
        Y = mulL(Xp)
    elif op == "Lt":
        Y = mulLt(Xp)
    elif op == "LLt":
        Z = mulLt(Xp)
        if F.kind == "ldlt":
            Z = Z * np.concatenate(F.d)[:, None]
        Y = mulL(Z)
    else:
        raise ValueError(op)
    return _from_perm(F, Y)


def flops_model(F: TLR, A: TLR, bs: int) -> dict:
    """Paper-model flop counts of the factorization F of A (per-tile chain of Equation 2)."""
    b, nb = F.b, F.nb
    out = dict(sample=0.0, project=0.0, diag=0.0, potrf=nb * b ** 3 / 3.0, trsm=0.0)
    for k in range(nb):
        for j in range(k):
            r = F.rank(k, j)
            out["diag"] += 4.0 * b * r * r + 2.0 * b * b * r
        for i in range(k + 1, nb):
            R = A.rank(i, k) + sum(F.rank(k, j) + F.rank(i, j) for j in range(k))
            t = max(F.rounds.get((i, k), 1), 1)
            r = F.rank(i, k)
            out["sample"] += 4.0 * b * bs * t * R
            out["project"] += 4.0 * b * r * R
            out["trsm"] += b * b * r
    out["total"] = sum(out.values())
    return out
