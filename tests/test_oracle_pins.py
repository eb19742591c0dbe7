"""Pins for the oracle: each test checks it against something other than itself
(published known answers, closed forms, library routines, Eckart-Young, brute force)."""
import math
import os

import numpy as np
import pytest

import inputs
from oracle import compress, dense, kdtree, kernel, measures, pcg, philox, tlr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(h, 16) for h in r]
        out = philox.philox4x32_10(np.array([v[:4]], dtype=np.uint64), (v[4], v[5]))
        assert [int(o) for o in out[0]] == v[6:10]


def test_omega_gaussian_statistics_and_layout():
    Om = philox.omega(7, 2, 3, 1, 256, 16)
    assert Om.shape == (256, 16)
    z = Om.ravel()
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1.0) < 0.05
    # column-major element order: a taller block shares its leading elements column by column
    Om2 = philox.omega(7, 2, 3, 1, 128, 32)
    assert np.array_equal(Om.T.ravel()[:4096], Om2.T.ravel()[:4096])
    # distinct rounds / columns / streams give independent blocks
    assert not np.allclose(Om, philox.omega(7, 2, 3, 2, 256, 16))
    assert not np.allclose(Om, philox.omega(7, 2, 4, 1, 256, 16))
    assert not np.allclose(Om, philox.omega(7, 1, 3, 1, 256, 16))


# ---------------------------------------------------------------- KD ordering
def test_kd_order_1d_is_sorted_order():
    x = inputs.points(1000, 1, 3)
    perm = kdtree.kd_order(x, 64)
    assert np.array_equal(perm, np.argsort(x[:, 0], kind="stable"))


@pytest.mark.parametrize("N,b,d", [(4096, 256, 2), (3000, 256, 3), (1000, 128, 2), (100, 128, 2)])
def test_kd_order_structure(N, b, d):
    x = inputs.points(N, d, 1)
    perm = kdtree.kd_order(x, b)
    assert np.array_equal(np.sort(perm), np.arange(N))

    def check(idx_ordered, n):
        if n <= b:
            return
        pts = x[idx_ordered]
        ext = pts.max(0) - pts.min(0)
        ax = int(np.argmax(ext))
        p = math.ceil(math.log2(n / b))
        nl = b * 2 ** (p - 1)
        left, right = idx_ordered[:nl], idx_ordered[nl:]
        assert x[left, ax].max() <= x[right, ax].min()
        check(left, nl)
        check(right, n - nl)

    check(perm, N)


# ---------------------------------------------------------------- dense factorizations
def _spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return M @ M.T + n * np.eye(n)


def test_cholesky_matches_lapack():
    A = _spd(60, 0)
    L = dense.cholesky(A)
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    assert np.allclose(L, np.tril(L))


def test_ldlt_closed_form_from_cholesky():
    A = _spd(50, 1)
    C = np.linalg.cholesky(A)
    L, d = dense.ldlt(A)
    assert np.allclose(d, np.diag(C) ** 2, rtol=1e-12)
    assert np.allclose(L, C / np.diag(C)[None, :], rtol=1e-11, atol=1e-12)
    assert np.allclose(np.diag(L), 1.0)


def test_ldlt_indefinite_without_pivoting():
    A = np.array([[2.0, 1.0, 0.0], [1.0, -3.0, 1.0], [0.0, 1.0, 4.0]])
    L, d = dense.ldlt(A)
    assert np.allclose(L @ np.diag(d) @ L.T, A, atol=1e-14)
    assert (d < 0).sum() == 1  # Sylvester's law of inertia: one negative eigenvalue
    assert (np.linalg.eigvalsh(A) < 0).sum() == 1


def test_cholesky_reports_failing_column():
    A = np.diag([1.0, 2.0, -1.0, 3.0])
    with pytest.raises(dense.NotPositiveDefinite) as ei:
        dense.cholesky(A)
    assert ei.value.index == 2


def test_triangular_solves_match_library():
    import scipy.linalg as sl
    A = _spd(40, 2)
    L = np.linalg.cholesky(A)
    B = np.random.default_rng(3).standard_normal((40, 3))
    assert np.allclose(dense.solve_lower(L, B), sl.solve_triangular(L, B, lower=True), rtol=1e-12)
    assert np.allclose(dense.solve_upper_t(L, B), sl.solve_triangular(L.T, B, lower=False), rtol=1e-12)
    Lu = np.tril(L, -1) + np.eye(40)
    assert np.allclose(dense.solve_lower(Lu, B, unit=True), sl.solve_triangular(Lu, B, lower=True, unit_diagonal=True))


# ---------------------------------------------------------------- compressors
def _low_rank(m, n, r, seed, decay=None):
    rng = np.random.default_rng(seed)
    X, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Y, _ = np.linalg.qr(rng.standard_normal((n, r)))
    s = np.ones(r) if decay is None else decay ** np.arange(r)
    return (X * s) @ Y.T, s


def test_svd_truncate_eckart_young():
    T, s = _low_rank(100, 80, 30, 0, decay=0.5)
    for eps in [1e-1, 1e-3, 1e-6]:
        Q, B = compress.svd_truncate(T, eps)
        r = Q.shape[1]
        assert r == int(np.sum(s > eps))
        err = np.linalg.norm(T - Q @ B.T, 2)
        assert err <= eps * (1 + 1e-8)
        assert abs(err - (s[r] if r < 30 else 0.0)) < 1e-12
        assert np.allclose(Q.T @ Q, np.eye(r), atol=1e-13)


def test_svd_truncate_exact_rank():
    T, _ = _low_rank(64, 64, 7, 1)
    Q, B = compress.svd_truncate(T, 1e-10)
    assert Q.shape[1] == 7


def test_chol_drop_keeps_rank_of_deficient_panel():
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((50, 3)) @ rng.standard_normal((3, 8))  # rank 3, 8 columns
    R, keep = compress.chol_drop(Y.T @ Y, 0.0)
    assert len(keep) == 3 and keep == [0, 1, 2]
    assert np.allclose(R.T @ R, (Y.T @ Y)[np.ix_(keep, keep)], rtol=1e-10)


@pytest.mark.parametrize("r,bs", [(5, 16), (16, 16), (40, 16), (70, 32)])
def test_ara_exact_rank_and_bound(r, bs):
    T, _ = _low_rank(256, 256, r, 5)
    om = lambda t: philox.omega(11, 9, 0, t, 256, bs)
    Q, B, t = compress.ara_dense(T, bs, 1e-8, om)
    assert Q.shape[1] == r  # exactly the rank of T: more columns would be noise below tau
    assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
    assert np.linalg.norm(T - Q @ B.T, 2) <= 1e-8


def test_ara_error_bound_holds_over_seeds():
    T, s = _low_rank(200, 200, 60, 6, decay=0.7)
    for seed in range(8):
        for eps in [1e-2, 1e-5, 1e-9]:
            Q, B, _ = compress.ara_dense(T, 16, eps, lambda t: philox.omega(seed, 9, 0, t, 200, 16))
            assert np.linalg.norm(T - Q @ B.T, 2) <= eps
            assert Q.shape[1] >= int(np.sum(s > eps))  # never below the optimal (SVD) rank


def test_ara_zero_tile_has_rank_zero():
    Q, B, t = compress.ara_dense(np.zeros((64, 64)), 16, 1e-6, lambda t: philox.omega(0, 9, 0, t, 64, 16))
    assert Q.shape == (64, 0) and t == 1


# ---------------------------------------------------------------- OU closed form (1D exponential kernel)
def _ou_closed_form(x, ell):
    """Exact Cholesky factor of exp(-|x_i - x_j|/ell) for sorted 1D x (Ornstein-Uhlenbeck covariance)."""
    n = len(x)
    s = np.ones(n)
    s[1:] = np.sqrt(1.0 - np.exp(-2.0 * np.diff(x) / ell))
    L = np.exp(-(x[:, None] - x[None, :]) / ell) * s[None, :]
    return np.tril(L), float(np.sum(np.log(1.0 - np.exp(-2.0 * np.diff(x) / ell))))


@pytest.mark.parametrize("compressor", ["svd", "ara"])
def test_tlr_ou_closed_form(compressor):
    N, b, ell = 512, 64, 0.3
    x = inputs.points(N, 1, 8)
    A = tlr.build(x, b, 1e-12, ell, 0.0, compressor=compressor, bs=8)
    xs = A.xo[:, 0]
    assert np.all(np.diff(xs) > 0)
    F = tlr.factor(A, 1e-12, compressor=compressor, bs=8)
    Lex, ld = _ou_closed_form(xs, ell)
    assert A.ranks()[np.tril_indices(A.nb, -1)].max() == 1  # every off-diagonal tile is rank 1
    lr = F.ranks()[np.tril_indices(F.nb, -1)]
    # SVD keeps sigma_2 <= eps: exact rank 1.  ARA tests against eps/(10 sqrt(2/pi)), so the
    # eps-level errors of earlier columns can add one direction to a tile.
    assert lr.max() == 1 if compressor == "svd" else (lr.max() <= 2 and lr.mean() < 1.5)
    assert np.allclose(F.to_dense(), Lex, atol=1e-9)
    assert abs(tlr.logdet(F) - ld) < 1e-8 * abs(ld)
    G = tlr.factor(A, 1e-12, ldl=True, compressor=compressor, bs=8)
    assert abs(tlr.logdet(G) - ld) < 1e-8 * abs(ld)


# ---------------------------------------------------------------- TLR oracle vs dense at tight eps
@pytest.mark.parametrize("N,b,d", [(1024, 128, 2), (1500, 256, 3)])
def test_tlr_matches_dense_at_tight_eps(N, b, d):
    ell, nug = (0.1 if d == 2 else 0.2), 1e-4
    x = inputs.points(N, d, 2)
    A = tlr.build(x, b, 1e-14, ell, nug)
    F = tlr.factor(A, 1e-14)
    Ad = kernel.dense(x, ell, nug)
    FF = tlr.matvec(F, np.eye(N), "LLt")
    assert np.linalg.norm(FF - Ad, 2) / np.linalg.norm(Ad, 2) < 1e-10
    s, ld = np.linalg.slogdet(Ad)
    assert s > 0 and abs(tlr.logdet(F) - ld) < 1e-10 * abs(ld)
    Y = inputs.rhs(N, 2, 4)
    assert np.allclose(tlr.solve(F, Y), np.linalg.solve(Ad, Y), rtol=1e-6, atol=1e-8 * np.abs(np.linalg.solve(Ad, Y)).max())
    G = tlr.factor(A, 1e-14, ldl=True)
    assert abs(tlr.logdet(G) - ld) < 1e-10 * abs(ld)
    # padded last tile (N not a multiple of b): padding rows of L are identity
    if N % b:
        Ld = F.to_dense()
        assert np.allclose(Ld[N:, N:], np.eye(F.nb * b - N))


def test_tlr_matvec_A_matches_dense():
    x = inputs.points(700, 2, 5)
    A = tlr.build(x, 128, 1e-12, 0.1, 1e-4)
    X = inputs.rhs(700, 3, 1)
    assert np.allclose(tlr.matvec(A, X, "A"), kernel.dense(x, 0.1, 1e-4) @ X, atol=1e-9)


# ---------------------------------------------------------------- invariants at working eps
def test_invariants_cov2d_small():
    N, b, eps = 2048, 256, 1e-6
    x = inputs.points(N, 2, 0)
    A = tlr.build(x, b, eps, 0.1, 1e-4)
    F = tlr.factor(A, eps)
    G = tlr.factor(A, eps, ldl=True)
    assert all(np.all(np.diag(L) > 0) for L in F.diag)
    assert all(np.all(dk > 0) for dk in G.d)
    low = F.ranks()[np.tril_indices(F.nb, -1)]
    assert low.max() <= b // 2
    Ad = kernel.dense(x, 0.1, 1e-4)
    x0 = inputs.start_vector(N)
    be = measures.backward_error(lambda v: Ad @ v, lambda v: tlr.matvec(F, v, "LLt")[:, 0], x0)
    assert be <= 10 * eps
    assert abs(tlr.logdet(F) - tlr.logdet(G)) <= 1e-3 * abs(tlr.logdet(F))


# ---------------------------------------------------------------- measures
def test_power_norm_diagonal():
    d = np.array([1.0, -7.0, 3.0, 0.5])
    assert abs(measures.power_norm(lambda v: d * v, np.ones(4), 200) - 7.0) < 1e-10


def test_backward_error_of_exact_factor_is_rounding_level():
    A = _spd(80, 9)
    L = np.linalg.cholesky(A)
    be = measures.backward_error(lambda v: A @ v, lambda v: L @ (L.T @ v), np.ones(80))
    assert be < 1e-14


def schur_pins_hold() -> bool:
    """Section 5.1.1 compensation (A_kk - D_k + diag(rowsum|D_k - Dbar_k|)), pinned without its formula:
    at eps = 1e-12 Dbar_k = D_k to rounding, so the factor is the uncompensated one; at eps = 1e-3 the
    first compensated column (k = 1, whose D_1 both factorizations share) changes L_11 L_11^T by a
    diagonal that is positive (the compensation is active) and, D-bar being an eps-truncation of the
    symmetric D_1, at most sqrt(b) eps per row (||E_i||_1 <= sqrt(b) ||E||_2 <= sqrt(b) eps)."""
    x = inputs.points(768, 2, 5)
    b = 128
    A = tlr.build(x, b, 1e-12, 0.1, 1e-4, compressor="svd")
    P, C = tlr.factor(A, 1e-12), tlr.factor(A, 1e-12, compensation="schur")
    for k in range(A.nb):
        if np.abs(P.diag[k] - C.diag[k]).max() > 1e-10 * np.abs(P.diag[k]).max():
            return False
    eps = 1e-3
    A = tlr.build(x, b, eps, 0.1, 1e-4, compressor="svd")
    try:
        P, C = tlr.factor(A, eps), tlr.factor(A, eps, compensation="schur")
    except dense.NotPositiveDefinite:
        return False
    if not np.array_equal(P.diag[0], C.diag[0]):
        return False
    D = C.diag[1] @ C.diag[1].T - P.diag[1] @ P.diag[1].T
    scale = np.abs(A.diag[1]).max()
    return (np.abs(D - np.diag(np.diag(D))).max() <= 1e-13 * scale and np.diag(D).min() > 0.0
            and np.diag(D).max() <= math.sqrt(b) * eps * (1 + 1e-12))


def test_schur_compensation_pins():
    assert schur_pins_hold()


def test_pcg_exact_preconditioner_converges_in_one_iteration():
    """With M = A the preconditioned residual is the error: one step solves the system."""
    rng = np.random.default_rng(3)
    G = rng.standard_normal((60, 60))
    A = G @ G.T + 60 * np.eye(60)
    b = rng.standard_normal((60, 2))
    x, it, res = pcg.pcg(lambda X: A @ X, lambda R: np.linalg.solve(A, R), b, 1e-12, 50)
    assert list(it) == [1, 1]
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-12 * np.abs(np.linalg.solve(A, b)).max())
    assert res.max() <= 1e-12


def test_pcg_terminates_in_as_many_steps_as_distinct_eigenvalues():
    """CG (M = I) on a matrix with 4 distinct eigenvalues: the Krylov space is exhausted after 4 steps."""
    d = np.repeat([1.0, 3.0, 10.0, 40.0], 20)
    A = np.diag(d)
    b = np.random.default_rng(4).standard_normal((80, 1))
    x, it, res = pcg.pcg(lambda X: A @ X, lambda R: R, b, 1e-10, 50)
    assert it[0] <= 4 and res[0] <= 1e-10
    assert np.allclose(x[:, 0], b[:, 0] / d, rtol=1e-9)


def test_pcg_matches_scipy_cg_and_handles_a_zero_column():
    """Against SciPy's CG with the same preconditioner, to the tolerance; a zero right-hand side takes 0 steps."""
    spla = pytest.importorskip("scipy.sparse.linalg")
    rng = np.random.default_rng(5)
    G = rng.standard_normal((70, 70))
    A = G @ G.T + np.eye(70)
    Md = np.diag(1.0 / np.diag(A))
    b = np.zeros((70, 2))
    b[:, 0] = rng.standard_normal(70)
    x, it, res = pcg.pcg(lambda X: A @ X, lambda R: Md @ R, b, 1e-11, 500)
    xs, info = spla.cg(A, b[:, 0], rtol=1e-13, maxiter=2000, M=Md)
    assert info == 0 and res[0] <= 1e-11 * 10
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x[:, 0] - xs) <= 1e-10 * cond * np.linalg.norm(xs)
    assert it[1] == 0 and not x[:, 1].any()


def _dense_block_pivoted_order(Ad: np.ndarray, b: int) -> list:
    """The definition of tile pivoting written densely: at each step the diagonal block of the current
    Schur complement with the largest Frobenius norm is moved to the front, then eliminated."""
    S = Ad.copy()
    nb = S.shape[0] // b
    order = list(range(nb))
    blk = lambda i: slice(i * b, (i + 1) * b)
    for k in range(nb):
        nrm = [np.linalg.norm(S[blk(i), blk(i)]) for i in range(k, nb)]
        p = k + int(np.argmax(nrm))
        if p != k:
            idx = np.arange(nb * b)
            idx[blk(k)], idx[blk(p)] = np.arange(p * b, (p + 1) * b), np.arange(k * b, (k + 1) * b)
            S = S[np.ix_(idx, idx)]
            order[k], order[p] = order[p], order[k]
        L = np.linalg.cholesky(S[blk(k), blk(k)])
        R = np.linalg.solve(L, S[blk(k), (k + 1) * b:]).T        # rows below, times L^-T
        S[(k + 1) * b:, (k + 1) * b:] -= R @ R.T
    return order


def pivoted_pins_hold() -> bool:
    """Algorithm 9 pinned: at eps = 1e-13 the pivoted TLR factor reproduces P A P^T, its solve and logdet
    those of the dense matrix, and its tile order is the dense block-pivoted Cholesky's."""
    x = inputs.points(1024, 2, 3)
    b = 128
    A = tlr.build(x, b, 1e-13, 0.1, 1e-4)
    try:
        F = tlr.factor_pivoted(A, 1e-13)
    except dense.NotPositiveDefinite:
        return False
    Ad = kernel.dense(x, 0.1, 1e-4)
    L = F.to_dense()
    P = F.perm
    if np.linalg.norm(L @ L.T - Ad[np.ix_(P, P)]) > 1e-10 * np.linalg.norm(Ad):
        return False
    Y = inputs.rhs(1024, 2, 5)
    Xd = np.linalg.solve(Ad, Y)
    if np.linalg.norm(tlr.solve(F, Y) - Xd) > 1e-9 * np.linalg.norm(Xd):
        return False
    if abs(tlr.logdet(F) - np.linalg.slogdet(Ad)[1]) > 1e-9 * abs(np.linalg.slogdet(Ad)[1]):
        return False
    Ako = Ad[np.ix_(A.perm, A.perm)]
    return list(F.tile_perm) == _dense_block_pivoted_order(Ako, b) and F.tile_perm != list(range(A.nb))


def test_pivoted_tlr_cholesky_pins():
    assert pivoted_pins_hold()


def test_pivoting_is_idle_when_updated_diagonal_tiles_decrease():
    """Tiles scaled by 4^-k: every updated diagonal tile is smaller than the one before, so no exchange
    happens and the pivoted factor is Algorithm 6's."""
    x = inputs.points(768, 2, 6)
    b = 128
    A = tlr.build(x, b, 1e-10, 0.1, 1e-4)
    s = 4.0 ** -np.arange(A.nb)
    A.diag = [A.diag[k] * s[k] ** 2 for k in range(A.nb)]
    for (i, j) in list(A.U):
        A.U[(i, j)] = A.U[(i, j)] * s[i]
        A.V[(i, j)] = A.V[(i, j)] * s[j]
    F = tlr.factor_pivoted(A, 1e-10)
    G = tlr.factor(A, 1e-10)
    assert F.tile_perm == list(range(A.nb))
    for k in range(A.nb):
        assert np.array_equal(F.diag[k], G.diag[k])
    for key in G.U:
        assert np.array_equal(F.U[key], G.U[key]) and np.array_equal(F.V[key], G.V[key])


def test_modified_cholesky_closed_forms():
    """Algorithm 8 with Cheng-Higham's modification: positive definite input -> plain Cholesky, E = 0;
    a diagonal input -> entries raised to delta; a 2x2 pivot block [[1,2],[2,1]] (eigenvalues 3, -1)
    -> the block with eigenvalues 3 and delta."""
    rng = np.random.default_rng(1)
    G = rng.standard_normal((20, 20))
    S = G @ G.T + np.eye(20)
    L, e = dense.modified_cholesky(S)
    Lr = np.linalg.cholesky(S)
    assert e == 0.0 and np.abs(L - Lr).max() <= 1e-13 * np.abs(Lr).max()
    a = np.array([3.0, -1.0, 2.0, -1e-12, 5.0])
    L, e = dense.modified_cholesky(np.diag(a), delta=1e-3)
    assert np.allclose(L @ L.T, np.diag(np.maximum(a, 1e-3)), rtol=1e-14, atol=0)
    assert abs(e - 1.001) <= 1e-12
    A = np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, -3.0]])
    dl = 1e-2
    L, e = dense.modified_cholesky(A, delta=dl)
    ref = np.zeros((3, 3))
    ref[:2, :2] = [[(3 + dl) / 2, (3 - dl) / 2], [(3 - dl) / 2, (3 + dl) / 2]]
    ref[2, 2] = dl
    assert np.allclose(L @ L.T, ref, rtol=0, atol=1e-14)


def modchol_pins_hold() -> bool:
    """In the TLR factorization (Algorithm 6 with Algorithm 8 for the diagonal tiles) the modification
    stays inside the tile it repaired: A - s I, made indefinite by s just above lambda_min(A), fails the
    plain factorization at tile t; with modified Cholesky L L^T equals A - s I everywhere except block
    (t, t), where the difference is the E of the modified Cholesky of that tile's exact Schur
    complement, and L L^T is positive definite."""
    x = inputs.points(768, 2, 9)
    b = 128
    Ad = kernel.dense(x, 0.1, 1e-4)
    sh = np.linalg.eigvalsh(Ad).min() + 1e-5
    A = tlr.build(x, b, 1e-12, 0.1, 1e-4 - sh)
    try:
        tlr.factor(A, 1e-12)
        return False
    except dense.NotPositiveDefinite as ex:
        t = ex.tile
    try:
        F = tlr.factor(A, 1e-12, compensation="modchol")
    except dense.NotPositiveDefinite:
        return False
    L = F.to_dense()
    As = (Ad - sh * np.eye(768))[np.ix_(F.perm, F.perm)]
    Dif = L @ L.T - As
    blk = slice(t * b, (t + 1) * b)
    off = Dif.copy()
    off[blk, blk] = 0.0
    n0 = t * b
    S = As[blk, blk] - As[blk, :n0] @ np.linalg.solve(As[:n0, :n0], As[:n0, blk]) if t else As[blk, blk]
    _, e = dense.modified_cholesky(S)
    return (np.abs(off).max() <= 1e-9 * np.abs(As).max() and e > 0
            and abs(np.linalg.norm(Dif[blk, blk], 2) - e) <= 1e-6 * e and np.linalg.eigvalsh(L @ L.T).min() > 0)


def test_modified_cholesky_in_tlr_factor_pins():
    assert modchol_pins_hold()


def test_trim_gives_the_truncated_svd_rank_and_error():
    """Trimming an ARA tile keeps exactly the ranks of the tile's own truncated SVD (Eckart-Young: the
    error is the first dropped singular value), and never more than ARA found."""
    x = inputs.points(512, 2, 7)
    xo = x[kdtree.kd_order(x, 128)]
    for (i, j) in [(1, 0), (3, 0), (2, 1)]:
        T = kernel.tile(xo, i, j, 128, 0.1, 1e-4)
        for eps in (1e-6, 1e-3):
            Q, B, _ = compress.ara_dense(T, 16, eps, lambda t: philox.omega(3, 1, 0, t, 128, 16))
            Qt, Bt = compress.trim(Q, B, eps)
            sv = np.linalg.svd(T, compute_uv=False)
            r_svd = int(np.count_nonzero(sv > eps))
            assert Qt.shape[1] <= Q.shape[1]
            assert abs(Qt.shape[1] - r_svd) <= 1          # the ARA basis captures T to ~eps / 10
            assert np.linalg.norm(T - Qt @ Bt.T, 2) <= 1.01 * eps
            assert np.allclose(Qt.T @ Qt, np.eye(Qt.shape[1]), atol=1e-12)


def trim_pins_hold(trim=None) -> bool:
    """Rank trimming pinned by a closed form: tiles with a prescribed spectrum (inputs.lowrank_tiles),
    eps halfway between two prescribed singular values.  The trimmed rank is exactly the number of
    values above eps, the kept singular values are the prescribed ones, the error is the first dropped
    value (Eckart-Young), and the new U has orthonormal columns."""
    trim = trim or compress.trim
    Q, B, s = inputs.lowrank_tiles(3, 96, 20, seed=11)
    step = 11.0 / 19
    for k in (4, 12):
        eps = 10.0 ** (1.0 - step * (k + 0.5))
        for t in range(3):
            Qt, Bt = trim(Q[t], B[t], eps)
            q = Qt.shape[1]
            if q != k + 1 or Bt.shape[1] != q:
                return False
            if not np.allclose(Qt.T @ Qt, np.eye(q), atol=1e-12):
                return False
            if not np.allclose(np.linalg.svd(Qt @ Bt.T, compute_uv=False)[:q], s[t][:q], rtol=1e-10, atol=0):
                return False
            if abs(np.linalg.norm(Q[t] @ B[t].T - Qt @ Bt.T, 2) - s[t][q]) > 1e-10 * s[t][q] + 1e-14:
                return False
    return True


def test_trim_matches_the_prescribed_spectrum():
    assert trim_pins_hold()


# Hand-computed kernel entries in 2D and 3D (Section 6: A_ij = exp(-||x_i - x_j||_2 / ell)): point
# pairs whose Euclidean distance is exact (3-4-5 and 1-2-2 triangles).  A wrong norm (L1, squared,
# max), a dropped coordinate or a swapped length scale gives a different value for at least one.
_KERNEL_PAIRS = [
    # (x_i, x_j, ell, exact distance)
    ((0.1, 0.2), (0.4, 0.6), 0.1, 0.5),
    ((0.75, 0.25), (0.75, 0.0), 0.1, 0.25),
    ((0.0, 0.0, 0.0), (0.1, 0.2, 0.2), 0.2, 0.3),
    ((0.5, 0.5, 0.5), (0.5, 0.8, 0.1), 0.2, 0.5),
    ((0.25, 0.5, 0.75), (0.25, 0.5, 0.75), 0.2, 0.0),
]


def test_kernel_entries_2d_3d_hand_computed():
    for xi, xj, ell, dist in _KERNEL_PAIRS:
        a = kernel.kernel_block(np.array([xi]), np.array([xj]), ell)[0, 0]
        assert a == pytest.approx(math.exp(-dist / ell), rel=4e-15, abs=0.0), (xi, xj)
    # the tile assembly puts the nugget on the diagonal only, and identity on padded rows
    x = np.array([[0.1, 0.2], [0.4, 0.6], [0.9, 0.9]])
    T = kernel.tile(x, 0, 0, 4, 0.1, 1e-4)
    assert T[0, 0] == 1.0 + 1e-4 and T[1, 1] == 1.0 + 1e-4 and T[3, 3] == 1.0
    assert T[0, 1] == T[1, 0] == pytest.approx(math.exp(-5.0), rel=4e-15)
    assert T[3, 0] == 0.0 and T[0, 3] == 0.0


def test_c_kernel_product_hand_computed_and_dense():
    """The plain-C exact product (used at full size) applied to unit vectors returns the hand-computed
    entries, and equals the dense matrix times a block of vectors."""
    from oracle import cmatvec
    for xi, xj, ell, dist in _KERNEL_PAIRS:
        x = np.array([xi, xj])
        col = cmatvec.matvec(x, ell, 1e-4, np.array([0.0, 1.0]))
        assert col[0] == pytest.approx(math.exp(-dist / ell), rel=4e-15)  # off the diagonal: no nugget
        assert col[1] == 1.0 + 1e-4
    x = inputs.points(300, 3, 11)
    X = np.random.default_rng(0).standard_normal((300, 5))
    Y = cmatvec.matvec(x, 0.2, 1e-4, X)
    R = kernel.dense(x, 0.2, 1e-4) @ X
    assert np.abs(Y - R).max() <= 1e-13 * np.abs(R).max()


def test_block_power_iteration_equals_single_and_converges():
    """measures.power_norms runs one independent power iteration per column: each column equals
    power_norm on its own operator, and both reach ||M||_2 of a symmetric matrix with a gap."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    Ms = [(Q * np.linspace(-s, 0.5 * s, 40)) @ Q.T for s in (1.0, 3.0, 0.0)]
    x0 = rng.standard_normal(40)
    lam = measures.power_norms(lambda V: np.stack([Ms[c] @ V[:, c] for c in range(3)], axis=1),
                               np.repeat(x0[:, None], 3, axis=1), iters=200)
    for c in range(3):
        assert lam[c] == pytest.approx(measures.power_norm(lambda v: Ms[c] @ v, x0, iters=200), rel=1e-14, abs=0.0)
    assert lam[0] == pytest.approx(1.0, rel=1e-8) and lam[1] == pytest.approx(3.0, rel=1e-8) and lam[2] == 0.0
