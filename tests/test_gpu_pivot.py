"""Tile-pivoted TLR Cholesky (Algorithm 9, Section 5.2) on the GPU (`opts.pivot = PIVOT_FROBENIUS`)
against the oracle's `tlr.factor_pivoted` with the same ARA (same Gaussian blocks): the same tile
exchanges (point order), ranks, factor tiles, logdet and solves; and against the definition, L L^T
= P A P^T with P the factor's point order."""
import numpy as np
import pytest

import inputs
from oracle import compress, kernel, tlr

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# nb = 8-16, 2D and 3D; every case exchanges tiles at most steps.  The smallest relative gap
# between the two largest updated-tile norms at any step (from the oracle) is 5.6e-4 or more, far above
# the difference rounding and eps-level compression can make, so the pivot order is unique.
CASES = {
    "cov2d_1k_b128": dict(N=1024, d=2, ell=0.1, nugget=1e-4, b=128, bs=16, seed=3, eps=1e-6),
    "cov2d_1536_b128": dict(N=1536, d=2, ell=0.1, nugget=1e-4, b=128, bs=16, seed=5, eps=1e-8),
    "cov3d_2k_b256": dict(N=2048, d=3, ell=0.2, nugget=1e-4, b=256, bs=32, seed=4, eps=1e-6),
    "cov2d_4k_b256": dict(N=4096, d=2, ell=0.1, nugget=1e-4, b=256, bs=16, seed=6, eps=1e-6),
    # tiles that are not a multiple of 16: FP64 products throughout (no chunk planes to exchange)
    "cov2d_1k_b100": dict(N=1000, d=2, ell=0.1, nugget=1e-4, b=100, bs=8, seed=7, eps=1e-6),
    "cov3d_1200_b120": dict(N=1200, d=3, ell=0.2, nugget=1e-4, b=120, bs=8, seed=2, eps=1e-6),
}


def _smallest_gap(Ao, eps, bs):
    """The oracle's pivoted factorization, recording the relative gap between the two largest
    updated-tile norms at each step."""
    gaps = []
    orig = tlr._select_pivot

    def sel(Ad, D, k):
        nrm = sorted((np.linalg.norm(Ad[i] - D[i]) for i in range(k, len(Ad))), reverse=True)
        if len(nrm) > 1:
            gaps.append((nrm[0] - nrm[1]) / nrm[0])
        return orig(Ad, D, k)
    tlr._select_pivot = sel
    try:
        Fo = tlr.factor_pivoted(Ao, eps, compressor="ara", bs=bs, seed=7)
    finally:
        tlr._select_pivot = orig
    return Fo, min(gaps)


@pytest.fixture(scope="module", params=list(CASES))
def case(request, T, ctx):
    w = CASES[request.param]
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=7))
    Ao = tlr.build(x, w["b"], w["eps"], w["ell"], w["nugget"], compressor="ara", bs=w["bs"], seed=7)
    Fo, gap = _smallest_gap(Ao, w["eps"], w["bs"])
    return dict(w=w, x=x, A=A, Ao=Ao, Fo=Fo, gap=gap)


def _popts(T, w, **kw):
    return T.default_opts(bs=w["bs"], seed=7, pivot=T.PIVOT_FROBENIUS, **kw)


def _tile_close(w, got, ref, t):
    """Rounding tolerance t (relative to the tile's largest entry, scaled by b / 256 above 256), or one
    ARA threshold: two eps-accurate ARA bases of inputs that differ by rounding may differ by that much
    in directions whose singular values lie near the threshold (the ranks still agree exactly)."""
    thr = w["eps"] / compress.HALKO
    tol = t * max(1.0, w["b"] / 256.0)
    return float(np.max(np.abs(got - ref))) <= max(tol * float(np.max(np.abs(ref))), thr)


def test_pivoted_factor_matches_oracle(T, ctx, case):
    w, Fo = case["w"], case["Fo"]
    assert case["gap"] > 1e-4 and Fo.tile_perm != list(range(Fo.nb))
    F = case["A"].copy()
    F.potrf(w["eps"], _popts(T, w))
    # the same exchanges: the factor's point order is the oracle's
    assert np.array_equal(F.perm(), Fo.perm)
    assert np.array_equal(F.ranks(), Fo.ranks())
    for k in range(Fo.nb):
        L, _ = F.tile(k, k)
        assert _tile_close(w, np.tril(L), Fo.diag[k], 1e-10), k
    for (i, j) in Fo.U:
        U, V = F.tile(i, j)
        ref = Fo.U[(i, j)] @ Fo.V[(i, j)].T
        if np.abs(ref).max() > 0:
            assert _tile_close(w, U @ V.T, ref, 1e-9), (i, j)
    ld, sg = F.logdet()
    assert sg == 1 and abs(ld - tlr.logdet(Fo)) <= 1e-10 * abs(tlr.logdet(Fo))
    # solves and products in the original point order
    Y = inputs.rhs(w["N"], 3, 11)
    Yt = _t(T, Y)
    F.solve(Yt)
    assert rel(Yt.cpu().numpy(), tlr.solve(Fo, Y)) < 1e-9
    Z = inputs.rhs(w["N"], 2, 12)
    Zt = _t(T, Z)
    for op, name in [(T.OP_L, "L"), (T.OP_LT, "Lt"), (T.OP_LLT, "LLt")]:
        assert rel(F.matvec(Zt, op).cpu().numpy(), tlr.matvec(Fo, Z, name)) < 1e-10


def test_pivoted_factor_reproduces_the_permuted_matrix(T, ctx):
    """The definition: L L^T = P A P^T (P = the factor's point order) to the compression accuracy,
    A^{-1} y from the factor equals the dense solve, logdet equals the dense one."""
    x = inputs.points(1024, 2, 3)
    b, eps = 128, 1e-10
    A = ctx.compress(x, b, eps, 0.1, 1e-4, T.default_opts(bs=16, seed=7))
    F = A.copy()
    F.potrf(eps, T.default_opts(bs=16, seed=7, pivot=T.PIVOT_FROBENIUS))
    nb = 1024 // b
    L = np.zeros((1024, 1024))
    for k in range(nb):
        L[k * b:(k + 1) * b, k * b:(k + 1) * b] = np.tril(F.tile(k, k)[0])
        for i in range(k + 1, nb):
            U, V = F.tile(i, k)
            L[i * b:(i + 1) * b, k * b:(k + 1) * b] = U @ V.T
    Ad = kernel.dense(x, 0.1, 1e-4)
    P = F.perm()
    assert not np.array_equal(P, A.perm())  # tiles were exchanged
    assert np.linalg.norm(L @ L.T - Ad[np.ix_(P, P)]) <= 1e-11 * np.linalg.norm(Ad)  # oracle: 4.3e-13
    y = inputs.rhs(1024, 1, 5)
    yt = _t(T, y)
    F.solve(yt)
    xd = np.linalg.solve(Ad, y)
    assert rel(yt.cpu().numpy(), xd) < 1e-9  # oracle: 9.7e-12
    ld, sg = F.logdet()
    assert sg == 1 and abs(ld - np.linalg.slogdet(Ad)[1]) <= 1e-12 * abs(np.linalg.slogdet(Ad)[1])


def test_pivoted_with_shift_matches_oracle(T, ctx):
    """TLR_COMP_SHIFT with pivoting factors A + s I: the oracle's pivoted factorization of the same
    matrix with s added to its diagonal tiles."""
    w = CASES["cov2d_1k_b128"]
    s = 1e-3
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=7))
    Ao = tlr.build(x, w["b"], w["eps"], w["ell"], w["nugget"], compressor="ara", bs=w["bs"], seed=7)
    Ao.diag = [t + s * np.eye(w["b"]) for t in Ao.diag]
    Fo, gap = _smallest_gap(Ao, w["eps"], w["bs"])
    assert gap > 1e-4
    F = A.copy()
    F.potrf(w["eps"], _popts(T, w, compensation=T.COMP_SHIFT, shift=s))
    assert np.array_equal(F.perm(), Fo.perm) and np.array_equal(F.ranks(), Fo.ranks())
    ld, _ = F.logdet()
    assert abs(ld - tlr.logdet(Fo)) <= 1e-10 * abs(tlr.logdet(Fo))


def test_pivoted_in_a_batch_is_bitwise_its_alone_result(T, ctx, case):
    """A pivoting matrix factored beside a non-pivoting one: both equal their alone factors bitwise."""
    w = case["w"]
    F1 = case["A"].copy()
    F1.potrf(w["eps"], _popts(T, w))
    G1 = case["A"].copy()
    G1.potrf(w["eps"], T.default_opts(bs=w["bs"], seed=7))
    F2, G2 = case["A"].copy(), case["A"].copy()
    st = ctx.factor_batch([F2, G2], w["eps"], [_popts(T, w), T.default_opts(bs=w["bs"], seed=7)])
    assert st == [T.OK, T.OK]
    for a, c in [(F1, F2), (G1, G2)]:
        assert np.array_equal(a.perm(), c.perm()) and np.array_equal(a.ranks(), c.ranks())
        nb = a.info()["nb"]
        for k in range(nb):
            assert np.array_equal(a.tile(k, k)[0], c.tile(k, k)[0])
            for i in range(k + 1, nb):
                for u, v in zip(a.tile(i, k), c.tile(i, k)):
                    assert np.array_equal(u, v)


def test_pivot_option_rules(T, ctx):
    x = inputs.points(1000, 2, 1)
    A = ctx.compress(x, 128, 1e-6, 0.1, 1e-4, T.default_opts(bs=16, seed=7))  # 1000 = 7 * 128 + 104
    C = ctx.compress(inputs.points(1024, 2, 1), 128, 1e-6, 0.1, 1e-4, T.default_opts(bs=16, seed=7))
    bad = [(A, dict()), (C, dict(precision=T.PREC_MIXED)), (C, dict(compensation=T.COMP_SCHUR)),
           (C, dict(compensation=T.COMP_MODCHOL)), (C, dict(pivot=2))]
    for M, kw in bad:
        o = T.default_opts(bs=16, seed=7, **({"pivot": T.PIVOT_FROBENIUS} | kw))
        with pytest.raises(T.TLRError) as ei:
            M.copy().potrf(1e-6, o)
        assert ei.value.status == T.ERR_ARG, kw
    with pytest.raises(T.TLRError) as ei:
        C.copy().ldlt(1e-6, T.default_opts(bs=16, seed=7, pivot=T.PIVOT_FROBENIUS))
    assert ei.value.status == T.ERR_ARG
