"""Modified Cholesky of an indefinite diagonal tile (Algorithm 8, Section 5.1.2): the GPU path
(`tlr_dense_modchol`, TLR_COMP_MODCHOL in the factorization) against the oracle's
`dense.modified_cholesky` (SciPy's Bunch-Kaufman LDL^T, Cheng-Higham modification) and its TLR
factorization with compensation "modchol"."""
import numpy as np
import pytest

import inputs
from oracle import dense, kernel, tlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import paper_2108_11932_gb300 as T
    T.build()
    return T


@pytest.fixture(scope="module")
def ctx(T):
    c = T.Context(0)
    yield c
    c.close()


def _t(T, A):
    import torch
    return T.fortran(torch.tensor(A, device="cuda:0"))


def _gpu_modchol(T, ctx, A):
    At = _t(T, A)
    mod, info = ctx.dense_modchol(At)
    return mod, info, np.tril(At.cpu().numpy())


def _indefinite(n, seed):
    """Q diag(lam) Q^T with lam ~ N(0, 1): about half the eigenvalues negative, many 2 x 2 pivots."""
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    return (Q * rng.standard_normal(n)) @ Q.T


CASES = {
    "indefinite_5": lambda: _indefinite(5, 1),
    "indefinite_64": lambda: _indefinite(64, 2),
    "indefinite_200": lambda: _indefinite(200, 3),  # past one 64-block, ragged
    "indefinite_513": lambda: _indefinite(513, 4),
    "diagonal": lambda: np.diag([3.0, -1.0, 2.0, -1e-12, 5.0]),
    "two_by_two_pivot": lambda: np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, -3.0]]),
    # a covariance tile shifted just below definiteness: one negative eigenvalue
    "shifted_covariance": lambda: (lambda K: K - (np.linalg.eigvalsh(K).min() + 1e-5) * np.eye(len(K)))(
        kernel.dense(inputs.points(256, 2, 5), 0.1, 1e-4)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_dense_modchol_matches_oracle(T, ctx, name):
    A = CASES[name]()
    n = len(A)
    mod, info, L = _gpu_modchol(T, ctx, A)
    Lo, eo = dense.modified_cholesky(A)
    assert mod == 1 and info == -1
    assert np.all(np.diag(L) > 0)
    S, So = L @ L.T, Lo @ Lo.T
    scale = np.abs(A).max()
    assert np.abs(S - So).max() <= 1e-11 * scale * max(1.0, n / 64.0), name
    # A + E is positive definite and E is the oracle's
    assert np.linalg.eigvalsh(S).min() > 0
    e = np.linalg.norm(S - A, 2)
    assert abs(e - eo) <= 1e-9 * max(eo, scale), (name, e, eo)


def test_dense_modchol_leaves_a_positive_definite_tile_to_cholesky(T, ctx):
    rng = np.random.default_rng(7)
    G = rng.standard_normal((96, 96))
    A = G @ G.T + np.eye(96)
    mod, info, L = _gpu_modchol(T, ctx, A)
    assert mod == 0 and info == -1
    Lr = np.linalg.cholesky(A)
    assert np.abs(L - Lr).max() <= 1e-12 * np.abs(Lr).max()


# the oracle pin's matrix: the 2D covariance shifted just below definiteness (one eigenvalue -1e-5), so
# that the plain TLR Cholesky breaks down at a diagonal tile
def _shifted_case():
    x = inputs.points(768, 2, 9)
    Ad = kernel.dense(x, 0.1, 1e-4)
    sh = np.linalg.eigvalsh(Ad).min() + 1e-5
    return x, 1e-4 - sh


@pytest.mark.parametrize("eps", [1e-10, 1e-6])
def test_tlr_modchol_matches_oracle(T, ctx, eps):
    x, nug = _shifted_case()
    b = 128
    o = T.default_opts(bs=16, seed=7)
    A = ctx.compress(x, b, eps, 0.1, nug, o)
    Ao = tlr.build(x, b, eps, 0.1, nug, compressor="ara", bs=16, seed=7)
    # without the safeguard the factorization stops at the oracle's failing tile
    with pytest.raises(dense.NotPositiveDefinite) as ex:
        tlr.factor(Ao, eps, compressor="ara", bs=16, seed=7)
    F0 = A.copy()
    with pytest.raises(T.TLRError) as ei:
        F0.potrf(eps, o)
    assert ei.value.status == T.ERR_NOT_SPD and F0.info()["k_fail"] == ex.value.tile
    # Algorithm 8 on that tile
    F = A.copy()
    F.potrf(eps, T.default_opts(bs=16, seed=7, compensation=T.COMP_MODCHOL))
    Fo = tlr.factor(Ao, eps, compressor="ara", bs=16, seed=7, compensation="modchol")
    assert np.array_equal(F.ranks(), Fo.ranks())
    thr = eps / 10.0 / np.sqrt(2.0 / np.pi)
    for k in range(Fo.nb):
        L, _ = F.tile(k, k)
        ref = Fo.diag[k]
        assert np.abs(np.tril(L) - ref).max() <= max(1e-9 * np.abs(ref).max(), thr), k
    for (i, j) in Fo.U:
        U, V = F.tile(i, j)
        ref = Fo.U[(i, j)] @ Fo.V[(i, j)].T
        if np.abs(ref).max() > 0:
            assert np.abs(U @ V.T - ref).max() <= max(1e-9 * np.abs(ref).max(), thr), (i, j)
    ld, sg = F.logdet()
    assert sg == 1 and abs(ld - tlr.logdet(Fo)) <= 1e-9 * abs(tlr.logdet(Fo))


def test_modchol_is_cholesky_only(T, ctx):
    x, nug = _shifted_case()
    A = ctx.compress(x, 128, 1e-6, 0.1, nug, T.default_opts(bs=16, seed=7))
    with pytest.raises(T.TLRError) as ei:
        A.copy().ldlt(1e-6, T.default_opts(bs=16, seed=7, compensation=T.COMP_MODCHOL))
    assert ei.value.status == T.ERR_ARG
