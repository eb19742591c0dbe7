"""ARA -> SVD rank trimming (Section 6) on the GPU: `tlr_trim_tiles` against the oracle's
`compress.trim` and the prescribed spectrum of synthetic tiles, and `tlr_trim` of compressed matrices
and factors against the exact kernel tiles and the dense matrix."""
import numpy as np
import pytest

import inputs
from oracle import compress, kdtree, kernel, tlr

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


def _dev_tiles(Q):
    """(ntiles, b, r) host blocks -> (ntiles, r, b) device tensor of column-major b x r blocks."""
    import torch
    return torch.tensor(np.ascontiguousarray(np.transpose(Q, (0, 2, 1))), device="cuda:0")


# (ntiles, b, r, k): eps halfway (geometrically) between the prescribed k-th and (k+1)-th singular
# values, 0.4 of a spectral step from every tile's values, so the kept rank is k + 1 for every tile
# (the last two: R^T in shared memory at r = 161, in global memory at b = 1024, r = 170)
TILE_CASES = [(6, 256, 40, 27), (4, 1024, 15, 9), (3, 512, 120, 100), (5, 100, 33, 0), (2, 64, 64, 63),
              (4, 128, 7, 6), (3, 200, 161, 120), (2, 1024, 170, 150)]


@pytest.mark.parametrize("nt,b,r,k", TILE_CASES)
def test_trim_tiles_match_the_oracle_and_the_prescribed_spectrum(T, ctx, nt, b, r, k):
    Q, B, s = inputs.lowrank_tiles(nt, b, r, seed=b + r)
    step = 11.0 / max(r - 1, 1)
    eps = 10.0 ** (1.0 - step * (k + 0.5)) if k < r - 1 else 1e-12
    Qo, Bo, rk = ctx.trim_tiles(_dev_tiles(Q), _dev_tiles(B), eps)
    Qo = np.transpose(Qo.cpu().numpy(), (0, 2, 1))
    Bo = np.transpose(Bo.cpu().numpy(), (0, 2, 1))
    for t in range(nt):
        want = int(np.count_nonzero(s[t] > eps))
        assert want == (k + 1 if k < r - 1 else r)
        Qt, Bt = compress.trim(Q[t], B[t], eps)
        assert rk[t] == want == Qt.shape[1], (t, rk[t], want)
        q = rk[t]
        assert not Qo[t][:, q:].any() and not Bo[t][:, q:].any()
        P, Pr = Qo[t][:, :q] @ Bo[t][:, :q].T, Qt @ Bt.T
        assert np.abs(P - Pr).max() <= 1e-12 * s[t][0], t
        assert np.abs(Qo[t][:, :q].T @ Qo[t][:, :q] - np.eye(q)).max() <= 1e-12
        # the kept singular values, in descending order, are the prescribed ones
        sv = np.linalg.norm(Bo[t][:, :q], axis=0)
        assert np.all(np.abs(sv - s[t][:q]) <= 1e-12 * s[t][0] + 1e-10 * s[t][:q])
        # the error is the first dropped singular value
        if q < r:
            e = np.linalg.norm(Q[t] @ B[t].T - P, 2)
            assert abs(e - s[t][q]) <= 1e-12 * s[t][0] + 1e-8 * s[t][q]


def test_trim_tiles_edge_cases(T, ctx):
    import torch
    Q, B, s = inputs.lowrank_tiles(2, 64, 8, seed=3)
    # eps above every singular value: rank 0, outputs zero
    Qo, Bo, rk = ctx.trim_tiles(_dev_tiles(Q), _dev_tiles(B), 1e3)
    assert list(rk) == [0, 0] and not Qo.any() and not Bo.any()
    # a zero tile
    Z = torch.zeros((1, 8, 64), dtype=torch.float64, device="cuda:0")
    Qo, Bo, rk = ctx.trim_tiles(_dev_tiles(Q[:1]), Z, 1e-12)
    assert list(rk) == [0]
    # a rank-deficient B (two equal columns): the zero singular value is dropped at any eps
    B2 = B[:1].copy()
    B2[0][:, 5] = B2[0][:, 4]
    sv = np.linalg.svd(B2[0], compute_uv=False)
    assert sv[-1] <= 1e-13 * sv[0] and sv[-2] > 1e-12
    Qo, Bo, rk = ctx.trim_tiles(_dev_tiles(Q[:1]), _dev_tiles(B2), 1e-12)
    assert rk[0] == 7 == compress.trim(Q[0], B2[0], 1e-12)[0].shape[1]


CASES = {
    "cov2d_2k_b256": dict(N=2048, d=2, ell=0.1, nugget=1e-4, b=256, bs=16, seed=0, eps=1e-6),
    "cov3d_ragged_b256": dict(N=1700, d=3, ell=0.2, nugget=1e-4, b=256, bs=32, seed=1, eps=1e-5),
    "cov2d_b100": dict(N=1000, d=2, ell=0.05, nugget=1e-4, b=100, bs=8, seed=4, eps=1e-7),
}


@pytest.mark.parametrize("name", list(CASES))
def test_trim_matrix_meets_the_threshold_with_the_svd_rank(T, ctx, name):
    """Every trimmed tile: rank within one of the exact tile's truncated-SVD rank, never above the ARA
    rank, error to the exact tile within 2 eps (ARA's eps plus the trim's), to the untrimmed tile within
    eps, orthonormal U."""
    w = CASES[name]
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=7))
    At = A.copy().trim(w["eps"])
    r0, r1 = A.ranks(), At.ranks()
    assert np.all(r1 <= r0) and r1.sum() < r0.sum()
    b, nb, N = w["b"], A.info()["nb"], w["N"]
    xo = x[kdtree.kd_order(x, b)]
    for i in range(nb):
        for j in range(i):
            U0, V0 = A.tile(i, j)
            U1, V1 = At.tile(i, j)
            assert U1.shape[1] == r1[i, j]
            Tx = kernel.tile(xo, i, j, b, w["ell"], w["nugget"])
            rs = int(np.count_nonzero(np.linalg.svd(Tx, compute_uv=False) > w["eps"]))
            assert abs(int(r1[i, j]) - rs) <= 1, (i, j, r1[i, j], rs)
            P1 = U1 @ V1.T
            assert np.linalg.norm(U0 @ V0.T - P1, 2) <= w["eps"] * (1 + 1e-6)
            assert np.linalg.norm(Tx - P1, 2) <= 2 * w["eps"]
            if r1[i, j]:
                assert np.abs(U1.T @ U1 - np.eye(r1[i, j])).max() <= 1e-12
    assert At.info()["bytes"] < A.info()["bytes"]
    # the trimmed matrix factors; with tiles truncated at eps (ARA's margin below eps removed) its solve
    # residual is that of the oracle's TLR built and recompressed by truncated SVDs, not the ARA path's
    Ad = kernel.dense(x, w["ell"], w["nugget"])
    y = inputs.rhs(N, 1, 5)
    res = []
    for M in (A, At):
        F = M.copy()
        F.potrf(w["eps"], T.default_opts(bs=w["bs"], seed=7))
        yt = _t(T, y)
        F.solve(yt)
        res.append(np.linalg.norm(Ad @ yt.cpu().numpy() - y) / np.linalg.norm(y))
    Fo = tlr.factor(tlr.build(x, b, w["eps"], w["ell"], w["nugget"]), w["eps"])
    res_svd = np.linalg.norm(Ad @ tlr.solve(Fo, y) - y) / np.linalg.norm(y)
    assert res[1] <= 2.0 * res_svd, (res, res_svd)


def test_trim_of_a_factor(T, ctx):
    """Trimming a factor changes each L(i,j) by at most eps in the 2-norm and leaves the diagonal tiles
    (so the log-determinant) unchanged."""
    w = CASES["cov2d_2k_b256"]
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=7))
    F = A.copy()
    F.potrf(w["eps"], T.default_opts(bs=w["bs"], seed=7))
    Ft = F.copy().trim(w["eps"])
    assert Ft.logdet() == F.logdet()
    nb = F.info()["nb"]
    for i in range(nb):
        for j in range(i):
            U0, V0 = F.tile(i, j)
            U1, V1 = Ft.tile(i, j)
            assert np.linalg.norm(U0 @ V0.T - U1 @ V1.T, 2) <= w["eps"] * (1 + 1e-6)
    y = inputs.rhs(w["N"], 2, 6)
    a, c = _t(T, y), _t(T, y)
    F.solve(a)
    Ft.solve(c)
    assert np.linalg.norm((a - c).cpu().numpy()) <= 1e-3 * np.linalg.norm(a.cpu().numpy())
