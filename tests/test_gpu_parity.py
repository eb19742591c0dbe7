"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Two oracles are used:
  * the oracle running the SAME algorithm (ARA with the same Philox Gaussian
    blocks, Algorithm 1/5/6/10): ranks are integers decided by the same
    threshold tests and must match exactly; factors agree to rounding;
  * the truncated-SVD oracle (the reference compressor): the acceptance rule
    backward error <= max(2x oracle's, 10 eps), solve residual <= 2x oracle's,
    |logdet - logdet_oracle| <= 1e-3 |logdet_oracle| at eps <= 1e-6.
Tolerances: FP64 everywhere; products of b x b operands accumulate O(b u)
rounding, the left-looking chain compounds it over nb columns, so factor
tiles are compared at 1e-10 relative to the tile's largest entry and
logdets at 1e-10 relative (ranks exactly) for b <= 256.  Dot-product and
Cholesky rounding bounds grow as gamma_n = n u with the contraction length
n = b (Higham, Accuracy and Stability, Sections 3.1 and 10.1), so for larger
tiles these rounding tolerances scale by b / 256 (`_tol`).
"""
import numpy as np
import pytest

import inputs
from oracle import pcg as opcg, compress, dense, kernel, measures, philox, tlr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import paper_2108_11932_gb300 as T
    T.build()
    return T


@pytest.fixture(scope="module")
def ctx(T):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return T.Context(0)


def _t(T, a):
    import torch
    return T.fortran(torch.tensor(np.asarray(a), device="cuda:0", dtype=torch.float64))


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------------ Omega
@pytest.mark.parametrize("seed,stream,k,t,b,bs", [(0, 1, 0, 0, 256, 16), (5, 2, 3, 7, 512, 32), (2**40 + 3, 3, 127, 9, 97, 5),
                                                  (1, 2, 0, 0, 1, 1)])
def test_omega_matches_oracle(T, ctx, seed, stream, k, t, b, bs):
    g = ctx.omega(seed, stream, k, t, b, bs).cpu().numpy()
    o = philox.omega(seed, stream, k, t, b, bs)
    assert g.shape == o.shape
    assert np.max(np.abs(g - o)) <= 1e-14 * max(1.0, np.max(np.abs(o)))


# ------------------------------------------------------------------ dense diagonal-tile kernels
@pytest.mark.parametrize("n", [1, 63, 64, 65, 200, 512, 1024])
def test_dense_potrf_ldlt_match_oracle(T, ctx, n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    At = _t(T, A)
    assert ctx.dense_potrf(At) == -1
    assert rel(np.tril(At.cpu().numpy()), dense.cholesky(A)) < 1e-12
    At = _t(T, A)
    assert ctx.dense_potrf(At, ldl=True) == -1
    Ld = At.cpu().numpy()
    Lo, do = dense.ldlt(A)
    assert rel(np.tril(Ld, -1) + np.eye(n), Lo) < 1e-12
    assert rel(np.diag(Ld), do) < 1e-12


def test_dense_potrf_reports_failing_column(T, ctx):
    n = 150
    A = np.eye(n) * 2.0
    A[97, 97] = -1.0
    At = _t(T, A)
    assert ctx.dense_potrf(At) == 97


def test_dense_ldlt_indefinite_pivot_free(T, ctx):
    rng = np.random.default_rng(3)
    n = 130
    M = rng.standard_normal((n, n))
    A = M + M.T + 0.1 * np.eye(n)  # indefinite, nonzero leading minors (generic)
    At = _t(T, A)
    assert ctx.dense_potrf(At, ldl=True) == -1
    Lo, do = dense.ldlt(A)
    Ld = At.cpu().numpy()
    assert rel(np.diag(Ld), do) < 1e-9
    assert (do < 0).any()


@pytest.mark.parametrize("n,nrhs,unit", [(300, 70, False), (64, 1, True), (1000, 5, False)])
def test_dense_trsm_matches_oracle(T, ctx, n, nrhs, unit):
    rng = np.random.default_rng(1)
    M = rng.standard_normal((n, n))
    L = np.linalg.cholesky(M @ M.T + n * np.eye(n))
    if unit:
        L = np.tril(L / np.diag(L)[None, :], -1) + np.eye(n)
    B = rng.standard_normal((n, nrhs))
    Lt, Bt = _t(T, L), _t(T, B)
    ctx.dense_trsm(Lt, Bt, unit=unit)
    assert rel(Bt.cpu().numpy(), dense.solve_lower(L, B, unit=unit)) < 1e-12


# ------------------------------------------------------------------ ARA on dense operands (Algorithm 1)
def _lowrank(n, r, seed, decay):
    rng = np.random.default_rng(seed)
    X, _ = np.linalg.qr(rng.standard_normal((n, r)))
    Y, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return (X * decay ** np.arange(r)) @ Y.T


# ------------------------------------------------------------------ split products (construction)
@pytest.mark.parametrize("n,ncols,trans,off", [(256, 16, 0, 1), (256, 37, 1, 3), (1024, 16, 0, 1),
                                               (512, 70, 1, 2), (64, 1, 0, 0), (256, 37, 2, 3), (1024, 16, 2, 1)])
def test_split_product_matches_fp64(T, ctx, n, ncols, trans, off):
    """T X and T^T X on the tcgen05 tensor cores by exact 7-bit splitting: error of an FP64 product.

    T is an exponential-kernel tile between two point clusters (entries over several orders of
    magnitude, off = 0: the diagonal tile with its nugget); X is Gaussian with one scaled column.
    The reference is numpy's FP64 product; the bound is a few units of 2^-53 of the block bounds
    times the sum of |X| over the inner dimension.
    """
    xo = inputs.points(n * (off + 1), 2, 11)
    Tn = kernel.tile(xo, off, 0, n, 0.1, 1e-4)
    X = inputs.gaussian(13, 2, n * ncols).reshape(ncols, n).T.copy()
    X[:, 0] *= 1e-9
    ref = (Tn.T if trans == 1 else Tn) @ X
    C = ctx.split_product(_t(T, Tn), _t(T, X), trans=trans).cpu().numpy()
    scale = np.abs(Tn).max() * np.abs(X).sum(axis=0)
    err = np.abs(C - ref) / scale[None, :]
    assert err.max() <= 8 * 2.0 ** -53, err.max()
    # the scaled column keeps its own accuracy (per-column bounds of X)
    assert np.abs(C[:, 0] - ref[:, 0]).max() <= 8 * 2.0 ** -53 * scale[0]


@pytest.mark.parametrize("d,ell", [(2, 0.1), (3, 0.2)])
def test_generated_tiles_match_oracle_entrywise(T, ctx, d, ell):
    """Diagonal tiles as generated (exp-kernel entries, nugget): a few units in the last place.

    exp(-r/ell) carries the rounding of its argument, relative error |r/ell| 2^-53 for either side,
    hence the bound grows with |log entry|.
    """
    from oracle import kdtree
    N, b = 1024, 256
    x = inputs.points(N, d, 21)
    A = ctx.compress(x, b, 1e-6, ell, 1e-4, T.default_opts(bs=16, seed=3))
    xo = x[kdtree.kd_order(x, b)]
    for k in range(N // b):
        got = A.tile(k, k)[0]
        ref = kernel.tile(xo, k, k, b, ell, 1e-4)
        bound = 4 * 2.0 ** -52 * (1.0 + np.abs(np.log(ref)))
        assert np.all(np.abs(got - ref) / np.abs(ref) <= bound)


@pytest.mark.parametrize("d,ell,shift,scale", [(1, 0.05, 0.0, 1.0), (2, 0.01, 0.0, 1.0), (3, 0.01, 0.0, 1.0),
                                               (2, 0.3, 1000.0, 7.0), (3, 0.2, -3.5, 1e-3)])
def test_generated_single_tile_all_distances(T, ctx, d, ell, shift, scale):
    """One tile holding every pair of 512 points: arguments |x_i - x_j|/ell from 0 (duplicated points)
    up to sqrt(d)/ell (173 at ell = 0.01 in 3D), and coordinates away from the unit box (shifted by
    1000, or scaled by 1e-3), all within a few units of 2^-52 (1 + |log entry|) of the oracle."""
    from oracle import kdtree
    N = 512
    x = inputs.points(N, d, 23) * scale + shift
    x[5] = x[17]
    x[300] = x[17]
    A = ctx.compress(x, N, 1e-6, ell * scale, 1e-4, T.default_opts(bs=16, seed=3))
    xo = x[kdtree.kd_order(x, N)]
    got = A.tile(0, 0)[0]
    ref = kernel.tile(xo, 0, 0, N, ell * scale, 1e-4)
    assert ref.min() < 1e-30 or ell >= 0.05
    bound = 4 * 2.0 ** -52 * (1.0 + np.abs(np.log(ref)))
    assert np.all(np.abs(got - ref) / np.abs(ref) <= bound)


def test_split_product_rejects_unaligned_size(T, ctx):
    Tn = np.eye(100)
    with pytest.raises(T.TLRError) as ei:
        ctx.split_product(_t(T, Tn), _t(T, np.ones((100, 2))))
    assert ei.value.status == T.ERR_LIMIT


@pytest.mark.parametrize("n", [256, 200])  # 200: row blocks and basis column blocks with ragged ends
def test_ara_dense_matches_oracle(T, ctx, n):
    import torch
    bs, eps = 16, 1e-6
    xo = inputs.points(2048, 2, 0)
    xo = xo[np.argsort(xo[:, 0])]
    ops = [kernel.tile(xo, 1, 0, n, 0.1, 1e-4), kernel.tile(xo, 5, 0, n, 0.1, 1e-4), np.zeros((n, n)),
           _lowrank(n, 7, 1, 1.0), _lowrank(n, 100, 2, 0.8), np.random.default_rng(5).standard_normal((n, n))]
    Tt = torch.tensor(np.stack([a.T for a in ops]), device="cuda:0")
    Q, B, r = ctx.ara_dense(Tt, bs, eps, seed=3, stream=1, k=0)
    for s, A in enumerate(ops):
        Qo, Bo, _ = compress.ara_dense(A, bs, eps, lambda t: philox.omega(3, 1, 0, t, n, bs))
        rg = int(r[s])
        assert rg == Qo.shape[1], (s, rg, Qo.shape[1])
        Qg, Bg = Q[s].cpu().numpy().T[:, :rg], B[s].cpu().numpy().T[:, :rg]
        if rg:
            assert rel(Qg @ Bg.T, Qo @ Bo.T) < 1e-10
            assert np.allclose(Qg.T @ Qg, np.eye(rg), atol=1e-12)
        assert np.linalg.norm(A - Qg @ Bg.T, 2) <= eps
    assert int(r[2]) == 0 and int(r[3]) == 7 and int(r[5]) == n


# ------------------------------------------------------------------ TLR: same algorithm as the oracle
CASES = {
    "cov2d_2k": dict(N=2048, d=2, ell=0.1, nugget=1e-4, b=256, bs=16, seed=0, eps=1e-6),
    "cov3d_ragged": dict(N=1700, d=3, ell=0.2, nugget=1e-4, b=256, bs=32, seed=1, eps=1e-5),  # nb = 7 (odd)
    "cov2d_b100": dict(N=1000, d=2, ell=0.05, nugget=1e-4, b=100, bs=8, seed=4, eps=1e-7),
    # the bench's tile shape (b = 1024, bs = 16: multi-round Gaussian-block ranges, long-K split-K
    # slices, Urow panels of ~1000 columns) at nb = 16, and C2's (b = 512, bs = 32) at eps = 1e-8
    "cov2d_16k_b1024": dict(N=16384, d=2, ell=0.1, nugget=1e-4, b=1024, bs=16, seed=2, eps=1e-6),
    "cov3d_4k_b512": dict(N=4096, d=3, ell=0.2, nugget=1e-4, b=512, bs=32, seed=1, eps=1e-8),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, T, ctx):
    w = CASES[request.param]
    x = inputs.points(w["N"], w["d"], w["seed"])
    o = T.default_opts(bs=w["bs"], seed=7)
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], o)
    Ao = tlr.build(x, w["b"], w["eps"], w["ell"], w["nugget"], compressor="ara", bs=w["bs"], seed=7)
    return dict(w=w, x=x, o=o, A=A, Ao=Ao, fo={})


def _tol(case, t):
    """Rounding tolerance t (set for b <= 256) scaled by b / 256 for larger tiles (gamma_b = b u)."""
    return t * max(1.0, case["w"]["b"] / 256.0)


def _tile_close(case, got, ref, t):
    """Factor tiles of two runs of the same ARA (identical ranks): max |got - ref| within the rounding
    tolerance t (relative to the tile's largest entry, scaled as in _tol) or within one ARA threshold
    eps / (10 sqrt(2/pi)), whichever is larger.  Two eps-accurate ARA approximations whose inputs differ
    by rounding are not rounding-close: directions whose singular values lie near the threshold enter
    both bases in rounding-dependent proportions, so the tiles may differ by up to the threshold (and the
    Schur compensation, a row sum of |D_k - Dbar_k|, by a few thresholds); the ranks must still agree
    exactly and logdet and solves stay at rounding level."""
    thr = case["w"]["eps"] / compress.HALKO
    return float(np.max(np.abs(got - ref))) <= max(_tol(case, t) * float(np.max(np.abs(ref))), thr)


def _oracle_factor(case, ldl, compensation=None):
    """The ARA oracle's factor of the case's matrix (same Gaussian blocks), computed once per case."""
    key = (ldl, compensation)
    if key not in case["fo"]:
        w = case["w"]
        case["fo"][key] = tlr.factor(case["Ao"], w["eps"], ldl=ldl, compressor="ara", bs=w["bs"], seed=7,
                                     compensation=compensation)
    return case["fo"][key]


def test_compress_matches_oracle_ara(case):
    A, Ao, w = case["A"], case["Ao"], case["w"]
    assert np.array_equal(A.perm(), Ao.perm)
    assert np.array_equal(A.ranks(), Ao.ranks())
    for k in range(Ao.nb):
        assert rel(A.tile(k, k)[0], Ao.diag[k]) < 1e-14
    for (i, j) in Ao.U:
        U, V = A.tile(i, j)
        ref = Ao.U[(i, j)] @ Ao.V[(i, j)].T
        if ref.size and np.abs(ref).max() > 0:
            assert rel(U @ V.T, ref) < _tol(case, 1e-10)
        assert np.linalg.norm(U @ V.T - kernel.tile(Ao.xo, i, j, w["b"], w["ell"], w["nugget"]), 2) <= w["eps"]


@pytest.mark.parametrize("ldl", [False, True])
def test_factor_matches_oracle_ara(case, ldl):
    w = case["w"]
    F = case["A"].copy()
    (F.ldlt if ldl else F.potrf)(w["eps"], case["o"])
    Fo = _oracle_factor(case, ldl)
    assert np.array_equal(F.ranks(), Fo.ranks())
    b = w["b"]
    for k in range(Fo.nb):
        L, d = F.tile(k, k)
        ref = Fo.diag[k]
        assert _tile_close(case, np.tril(L, -1) + (np.eye(b) if ldl else np.diag(np.diag(L))), ref, 1e-10)
        if ldl:
            assert _tile_close(case, d, Fo.d[k], 1e-10)
    for (i, j) in Fo.U:
        U, V = F.tile(i, j)
        ref = Fo.U[(i, j)] @ Fo.V[(i, j)].T
        if np.abs(ref).max() > 0:
            assert _tile_close(case, U @ V.T, ref, 1e-9)
    ld, sg = F.logdet()
    assert sg == 1 and abs(ld - tlr.logdet(Fo)) <= _tol(case, 1e-10) * abs(tlr.logdet(Fo))
    # solve and products against the oracle's factor
    Y = inputs.rhs(w["N"], 3, 11)
    import paper_2108_11932_gb300 as TT
    Yt = _t(TT, Y)
    F.solve(Yt)
    assert rel(Yt.cpu().numpy(), tlr.solve(Fo, Y)) < _tol(case, 1e-9)
    Z = inputs.rhs(w["N"], 2, 12)
    Zt = _t(TT, Z)
    for op, name in [(TT.OP_L, "L"), (TT.OP_LT, "Lt"), (TT.OP_LLT, "LLt")]:
        assert rel(F.matvec(Zt, op).cpu().numpy(), tlr.matvec(Fo, Z, name)) < _tol(case, 1e-10)


@pytest.mark.parametrize("ldl", [False, True])
def test_schur_compensation_matches_oracle_ara(case, ldl):
    """Section 5.1.1 compensation on both sides with one reading (Dbar_k from an ARA eps-basis of D_k
    drawn from the Schur Gaussian stream): identical ranks, factor tiles and logdet as the oracle's."""
    import paper_2108_11932_gb300 as TT
    w = case["w"]
    o = TT.default_opts(bs=w["bs"], seed=7, compensation=TT.COMP_SCHUR)
    F = case["A"].copy()
    (F.ldlt if ldl else F.potrf)(w["eps"], o)
    Fo = _oracle_factor(case, ldl, "schur")
    assert np.array_equal(F.ranks(), Fo.ranks())
    b = w["b"]
    for k in range(Fo.nb):
        L, d = F.tile(k, k)
        ref = Fo.diag[k]
        assert _tile_close(case, np.tril(L, -1) + (np.eye(b) if ldl else np.diag(np.diag(L))), ref, 1e-10)
        if ldl:
            assert _tile_close(case, d, Fo.d[k], 1e-10)
    for (i, j) in Fo.U:
        U, V = F.tile(i, j)
        ref = Fo.U[(i, j)] @ Fo.V[(i, j)].T
        if np.abs(ref).max() > 0:
            assert _tile_close(case, U @ V.T, ref, 1e-9)
    ld, _ = F.logdet()
    assert abs(ld - tlr.logdet(Fo)) <= _tol(case, 1e-10) * abs(tlr.logdet(Fo))
    F.free()


@pytest.mark.parametrize("ldl", [False, True])
def test_repeated_solves_replay_a_captured_graph(case, ldl):
    """A factor's solves with one nrhs: the first runs the plan's launches directly, the second captures
    them as a CUDA graph and replays it, later ones replay; every result matches the oracle's solve
    and the direct and replayed runs agree bitwise.  nrhs = 40 runs as groups of 32 and 8."""
    import paper_2108_11932_gb300 as TT
    w = case["w"]
    F = case["A"].copy()
    (F.ldlt if ldl else F.potrf)(w["eps"], case["o"])
    Fo = _oracle_factor(case, ldl)
    for nrhs in (1, 3, 40):
        Y = inputs.rhs(w["N"], nrhs, 20 + nrhs)
        ref = tlr.solve(Fo, Y)
        outs = []
        for rep in range(3):
            Yt = _t(TT, Y)
            l0 = F.ctx.launches()
            F.solve(Yt)
            assert F.ctx.launches() > l0  # replays count the graph's kernels
            outs.append(Yt.cpu().numpy())
            assert rel(outs[-1], ref) < _tol(case, 1e-9), (nrhs, rep)
        assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    F.free()


def test_tlr_product_of_A(case):
    import paper_2108_11932_gb300 as TT
    w = case["w"]
    Z = inputs.rhs(w["N"], 2, 13)
    assert rel(case["A"].matvec(_t(TT, Z), TT.OP_A).cpu().numpy(), tlr.matvec(case["Ao"], Z, "A")) < _tol(case, 1e-12)


def test_kernel_matvec_matches_oracle(T, ctx):
    x = inputs.points(3000, 3, 9)
    Z = inputs.rhs(3000, 5, 3)
    g = ctx.kernel_matvec(x, 0.2, 1e-4, _t(T, Z)).cpu().numpy()
    assert rel(g, kernel.matvec(x, 0.2, 1e-4, Z)) < 1e-13


# ------------------------------------------------------------------ dynamic batching, determinism
def test_batch_width_does_not_change_results(T, ctx):
    w = CASES["cov2d_2k"]
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=7))
    outs = []
    for slots in [0, 1, 3]:
        F = A.copy()
        F.potrf(w["eps"], T.default_opts(bs=w["bs"], seed=7, max_slots=slots))
        outs.append((F.ranks(), F.tile(5, 2), F.tile(7, 7)[0], F.logdet()[0]))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.array_equal(o[1][0], outs[0][1][0]) and np.array_equal(o[1][1], outs[0][1][1])
        assert np.array_equal(o[2], outs[0][2]) and o[3] == outs[0][3]


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("N,b", [(100, 128), (129, 128), (256, 128), (1, 16)])
def test_small_and_ragged_sizes_against_dense(T, ctx, N, b):
    x = inputs.points(N, 2, 21)
    A = ctx.compress(x, b, 1e-12, 0.1, 1e-2, T.default_opts(bs=8))
    F = A.copy().potrf(1e-12, T.default_opts(bs=8))
    Ad = kernel.dense(x, 0.1, 1e-2)
    s, ld = np.linalg.slogdet(Ad)
    assert abs(F.logdet()[0] - ld) <= 1e-9 * max(1.0, abs(ld))
    Y = inputs.rhs(N, 2, 1)
    Yt = _t(T, Y)
    F.solve(Yt)
    assert rel(Yt.cpu().numpy(), np.linalg.solve(Ad, Y)) < 1e-6


def test_not_positive_definite_is_reported(T, ctx):
    w = CASES["cov2d_2k"]
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=16))
    F = A.copy()
    bad = T.default_opts(bs=16, compensation=T.COMP_SHIFT, shift=-5.0)  # A - 5 I is indefinite
    with pytest.raises(T.TLRError) as ei:
        F.potrf(w["eps"], bad)
    assert ei.value.status == T.ERR_NOT_SPD
    inf = F.info()
    assert inf["state"] == 3 and inf["k_fail"] == 0
    with pytest.raises(T.TLRError) as ei:
        F.logdet()
    assert ei.value.status == T.ERR_STATE
    # the pivot-free LDL^T of the same indefinite matrix runs through (Section 5.3)
    G = A.copy()
    G.ldlt(w["eps"], bad)
    ld, sg = G.logdet()
    Go = tlr.factor(tlr.build(x, w["b"], w["eps"], w["ell"], w["nugget"], compressor="ara", bs=16, seed=0),
                    w["eps"], ldl=True, compressor="ara", bs=16, seed=0, compensation="shift", shift=-5.0)
    assert abs(ld - tlr.logdet(Go)) <= 1e-9 * abs(tlr.logdet(Go))
    assert sg == (-1 if sum(int(np.sum(dk < 0)) for dk in Go.d) % 2 else 1)


def test_invalid_arguments(T, ctx):
    x = inputs.points(100, 2, 0)
    with pytest.raises(T.TLRError) as ei:
        ctx.compress(x, 64, -1.0, 0.1, 1e-4)
    assert ei.value.status == T.ERR_ARG
    with pytest.raises(T.TLRError):
        ctx.compress(x, 64, 1e-6, 0.1, 1e-4, T.default_opts(bs=65))
    A = ctx.compress(x, 64, 1e-6, 0.1, 1e-4)
    with pytest.raises(T.TLRError) as ei:
        A.solve(_t(T, np.zeros((100, 1))))
    assert ei.value.status == T.ERR_STATE


# ------------------------------------------------------------------ acceptance vs the SVD oracle
def _gpu_backward_error(T, ctx, F, x, ell, nug, iters=30):
    import torch
    v0 = inputs.start_vector(x.shape[0])

    def EA(v):
        vt = torch.tensor(v, device="cuda:0")
        return ctx.kernel_matvec(x, ell, nug, vt).cpu().numpy()

    def EF(v):
        vt = torch.tensor(v, device="cuda:0")
        return F.matvec(vt).cpu().numpy()
    return measures.backward_error(EA, EF, v0, iters)


@pytest.mark.parametrize("ldl", [False, True])
def test_acceptance_cov2d_4k_against_svd_oracle(T, ctx, ldl):
    w = inputs.WORKLOADS["cov2d_4k"]
    eps = 1e-6
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], eps, w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=0))
    F = A.copy()
    (F.ldlt if ldl else F.potrf)(eps, T.default_opts(bs=w["bs"], seed=0))
    Ao = tlr.build(x, w["b"], eps, w["ell"], w["nugget"])
    Fo = tlr.factor(Ao, eps, ldl=ldl)
    Ad = kernel.dense(x, w["ell"], w["nugget"])
    v0 = inputs.start_vector(w["N"])
    be_o = measures.backward_error(lambda v: Ad @ v, lambda v: tlr.matvec(Fo, v, "LLt")[:, 0], v0)
    be_g = _gpu_backward_error(T, ctx, F, x, w["ell"], w["nugget"])
    assert be_g <= max(2 * be_o, 10 * eps), (be_g, be_o)
    Y = inputs.rhs(w["N"], 4, 5)
    Yt = _t(T, Y)
    F.solve(Yt)
    res_g = measures.residual(lambda Z: Ad @ Z, Yt.cpu().numpy(), Y)
    res_o = measures.residual(lambda Z: Ad @ Z, tlr.solve(Fo, Y), Y)
    assert res_g <= 2 * res_o, (res_g, res_o)
    ld_o = tlr.logdet(Fo)
    assert abs(F.logdet()[0] - ld_o) <= 1e-3 * abs(ld_o)


# ------------------------------------------------------------------ mixed precision (FP32 sampling chains)
@pytest.mark.parametrize("eps,ldl,prec", [(1e-2, False, 1), (1e-4, False, 1), (1e-4, True, 1),
                                          (1e-2, False, 2), (1e-4, False, 2), (1e-4, True, 2), (1e-2, True, 2)])
def test_mixed_precision_meets_acceptance(T, ctx, eps, ldl, prec):
    """Mixed sampling/projection products (FP64 orthogonalization, potrf, trsm) meet the same acceptance
    rule as the FP64 path: FP32 chains (prec 1) or products truncated to fewer 7-bit planes on the
    16-bit tensor cores (prec 2; the construction truncates too)."""
    w = inputs.WORKLOADS["cov2d_4k"]
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], eps, w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=0, precision=prec))
    F32 = A.copy()
    (F32.ldlt if ldl else F32.potrf)(eps, T.default_opts(bs=w["bs"], seed=0, precision=prec))
    F64 = A.copy()
    (F64.ldlt if ldl else F64.potrf)(eps, T.default_opts(bs=w["bs"], seed=0))
    Ao = tlr.build(x, w["b"], eps, w["ell"], w["nugget"])
    Fo = tlr.factor(Ao, eps, ldl=ldl)
    Ad = kernel.dense(x, w["ell"], w["nugget"])
    v0 = inputs.start_vector(w["N"])
    be_o = measures.backward_error(lambda v: Ad @ v, lambda v: tlr.matvec(Fo, v, "LLt")[:, 0], v0)
    be_32 = _gpu_backward_error(T, ctx, F32, x, w["ell"], w["nugget"])
    assert be_32 <= max(2 * be_o, 10 * eps), (be_32, be_o)
    Y = inputs.rhs(w["N"], 2, 5)
    Yt = _t(T, Y)
    F32.solve(Yt)
    res_32 = measures.residual(lambda Z: Ad @ Z, Yt.cpu().numpy(), Y)
    res_o = measures.residual(lambda Z: Ad @ Z, tlr.solve(Fo, Y), Y)
    assert res_32 <= 2 * res_o, (res_32, res_o)
    # error of the mixed path against the FP64 path on the same input (stated, bounded)
    ld32, ld64 = F32.logdet()[0], F64.logdet()[0]
    assert abs(ld32 - ld64) <= 1e-3 * abs(ld64)


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_falls_back_to_fp64_below_1e4(T, ctx, prec):
    w = CASES["cov2d_2k"]
    x = inputs.points(w["N"], w["d"], w["seed"])
    A = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=7))
    Am = ctx.compress(x, w["b"], w["eps"], w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=7, precision=prec))
    assert np.array_equal(A.ranks(), Am.ranks())
    F32 = Am.copy().potrf(w["eps"], T.default_opts(bs=w["bs"], seed=7, precision=prec))
    F64 = A.copy().potrf(w["eps"], T.default_opts(bs=w["bs"], seed=7))
    assert np.array_equal(F32.ranks(), F64.ranks())
    assert F32.logdet()[0] == F64.logdet()[0]


def test_truncated_planes_are_chosen_per_block_within_the_bound(T, ctx):
    """The mixed path's products use fewer 7-bit planes at eps = 1e-2 than at 1e-4, never fewer than 2,
    and every block of an FP64 run uses all 8 (tlr_split_planes); the mixed construction's tiles
    stay within eps of the FP64 construction's in 2-norm."""
    w = inputs.WORKLOADS["cov2d_4k"]
    x = inputs.points(w["N"], w["d"], w["seed"])
    used = {}
    for eps, prec in [(1e-2, 2), (1e-4, 2), (1e-2, 0)]:
        ctx.split_planes(reset=True)
        A = ctx.compress(x, w["b"], eps, w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=0, precision=prec))
        A.copy().potrf(eps, T.default_opts(bs=w["bs"], seed=0, precision=prec))
        c, _ = ctx.split_planes(reset=True)
        used[(eps, prec)] = c
        if prec == 2 and eps == 1e-2:
            Am = A
    assert sum(used[(1e-2, 0)][1:8]) == 0 and used[(1e-2, 0)][8] > 0
    mean = lambda c: sum(i * c[i] for i in range(9)) / max(sum(c), 1)
    assert used[(1e-2, 2)][1] == 0 and mean(used[(1e-2, 2)]) < mean(used[(1e-4, 2)]) < 8
    A64 = ctx.compress(x, w["b"], 1e-2, w["ell"], w["nugget"], T.default_opts(bs=w["bs"], seed=0))
    for (i, j) in [(1, 0), (5, 2), (15, 0)]:
        U, V = Am.tile(i, j)
        U6, V6 = A64.tile(i, j)
        assert np.linalg.norm(U @ V.T - U6 @ V6.T, 2) <= 2e-2


# ------------------------------------------------------------------ batched factorization of many matrices
BATCH = [dict(N=1500, d=2, ell=0.1, b=256, eps=1e-6, seed=31), dict(N=2048, d=3, ell=0.2, b=256, eps=1e-4, seed=32),
         dict(N=700, d=2, ell=0.05, b=128, eps=1e-7, seed=33), dict(N=1024, d=3, ell=0.3, b=128, eps=1e-5, seed=34),
         dict(N=1350, d=2, ell=0.15, b=256, eps=1e-6, seed=35)]  # nb = 6, 8, 6, 8, 6 (7 tiles when padded: 1350/256)


def _batch_inputs(T, ctx, specs, prec=0):
    mats, eps, opts = [], [], []
    for sp in specs:
        x = inputs.points(sp["N"], sp["d"], sp["seed"])
        o = T.default_opts(bs=16, seed=sp["seed"], precision=prec)
        mats.append(ctx.compress(x, sp["b"], sp["eps"], sp["ell"], 1e-4, o))
        eps.append(sp["eps"])
        opts.append(o)
    return mats, eps, opts


@pytest.mark.parametrize("ldl", [False, True])
def test_batch_equals_individual_bitwise(T, ctx, ldl):
    """A matrix factored inside a batch gives bit-identical factors to the same matrix alone."""
    mats, eps, opts = _batch_inputs(T, ctx, BATCH)
    alone = []
    for A, e, o in zip(mats, eps, opts):
        F = A.copy()
        (F.ldlt if ldl else F.potrf)(e, o)
        alone.append(F)
    batch = [A.copy() for A in mats]
    st = ctx.factor_batch(batch, eps, opts, ldl=ldl)
    assert st == [0] * len(batch)
    for F, G in zip(alone, batch):
        assert np.array_equal(F.ranks(), G.ranks())
        assert F.logdet() == G.logdet()
        nb = F.info()["nb"]
        for (i, j) in [(nb - 1, 0), (nb - 1, nb - 2), (1, 0)]:
            if i > j:
                a, g = F.tile(i, j), G.tile(i, j)
                assert np.array_equal(a[0], g[0]) and np.array_equal(a[1], g[1])
        assert np.array_equal(F.tile(nb - 1, nb - 1)[0], G.tile(nb - 1, nb - 1)[0])


def test_batch_matches_oracle(T, ctx):
    mats, eps, opts = _batch_inputs(T, ctx, BATCH)
    st = ctx.factor_batch(mats, eps, opts)
    assert st == [0] * len(mats)
    for sp, F in zip(BATCH, mats):
        x = inputs.points(sp["N"], sp["d"], sp["seed"])
        Ao = tlr.build(x, sp["b"], sp["eps"], sp["ell"], 1e-4, compressor="ara", bs=16, seed=sp["seed"])
        Fo = tlr.factor(Ao, sp["eps"], compressor="ara", bs=16, seed=sp["seed"])
        assert np.array_equal(F.ranks(), Fo.ranks())
        assert abs(F.logdet()[0] - tlr.logdet(Fo)) <= 1e-10 * abs(tlr.logdet(Fo))


def test_batch_isolates_a_failing_matrix(T, ctx):
    mats, eps, opts = _batch_inputs(T, ctx, BATCH)
    ref = []
    for A, e, o in zip(mats, eps, opts):
        ref.append(A.copy().potrf(e, o).logdet()[0])
    bad = T.default_opts(bs=16, seed=BATCH[1]["seed"], compensation=T.COMP_SHIFT, shift=-5.0)
    opts2 = list(opts)
    opts2[1] = bad
    st = ctx.factor_batch(mats, eps, opts2)
    assert st[1] == T.ERR_NOT_SPD and mats[1].info()["state"] == 3
    for m in (0, 2, 3):
        assert st[m] == 0 and mats[m].logdet()[0] == ref[m]


def test_batch_mixed_precision(T, ctx):
    specs = [dict(s, eps=1e-2) for s in BATCH]
    mats, eps, opts = _batch_inputs(T, ctx, specs, prec=1)
    alone = [A.copy().potrf(e, o) for A, e, o in zip(mats, eps, opts)]
    st = ctx.factor_batch(mats, eps, opts)
    assert st == [0] * len(mats)
    for F, G in zip(alone, mats):
        assert np.array_equal(F.ranks(), G.ranks()) and F.logdet() == G.logdet()


# ------------------------------------------------------------------ continuous batching (session)
def test_session_join_mid_flight_is_bitwise_identical(T, ctx):
    mats, eps, opts = _batch_inputs(T, ctx, BATCH)
    alone = [A.copy().potrf(e, o) for A, e, o in zip(mats, eps, opts)]
    S = T.Session(ctx)
    tickets = {0: S.add(mats[0], eps[0], opts[0])}
    S.step()
    S.step()
    tickets[1] = S.add(mats[1], eps[1], opts[1])   # joins while matrix 0 is at column 2
    S.step()
    tickets[2] = S.add(mats[2], eps[2], opts[2])
    tickets[3] = S.add(mats[3], eps[3], opts[3])
    while S.step():
        pass
    for m, t in tickets.items():
        done, st = S.poll(t)
        assert done and st == 0
        assert np.array_equal(alone[m].ranks(), mats[m].ranks())
        assert alone[m].logdet() == mats[m].logdet()
        nb = mats[m].info()["nb"]
        a, g = alone[m].tile(nb - 1, 0), mats[m].tile(nb - 1, 0)
        assert np.array_equal(a[0], g[0]) and np.array_equal(a[1], g[1])
    S.close()


def test_autotune_picks_a_measured_configuration(T, ctx):
    """The tuner times every configuration it may pick and returns the fastest of its coordinate search."""
    from paper_2108_11932_gb300 import autotune
    res = autotune.tune(ctx, dims=(2,), sizes=(2048,), candidates=(128, 256), bs_candidates=(16, 32),
                        width_candidates=(0, 8), repeats=1)
    b, bs, width = res["table"][(2, 11)]
    tm = res["timings"]
    assert (2, 2048, b, bs, width) in tm
    # each coordinate is the fastest measured along its line
    assert tm[(2, 2048, b, 16, 0)] == min(tm[(2, 2048, v, 16, 0)] for v in (128, 256))
    assert tm[(2, 2048, b, bs, 0)] == min(tm[(2, 2048, b, v, 0)] for v in (16, 32))
    assert tm[(2, 2048, b, bs, width)] == min(tm[(2, 2048, b, bs, v)] for v in (0, 8))


def test_pcg_matches_oracle(T, ctx):
    """Section 6's use of a low-accuracy factor: PCG on the eps = 1e-8 compressed covariance matrix,
    preconditioned by the factor of the eps = 1e-3 one with the shift eps I, against the oracle's PCG on
    the oracle's matrices (same ARA streams): iteration counts within one of each other, true residuals
    at the tolerance, a zero right-hand side solved by x = 0 in 0 iterations, and far fewer iterations
    than unpreconditioned CG would need."""
    N, d, ell, nug, b, bs, tol = 2048, 2, 0.1, 1e-4, 256, 16, 1e-8
    x = inputs.points(N, d, 0)
    o = T.default_opts(bs=bs, seed=7)
    A = ctx.compress(x, b, 1e-8, ell, nug, o)
    Fm = ctx.compress(x, b, 1e-3, ell, nug, o)
    Fm.potrf(1e-3, T.default_opts(bs=bs, seed=7, compensation=T.COMP_SHIFT, shift=1e-3))
    Ao = tlr.build(x, b, 1e-8, ell, nug, compressor="ara", bs=bs, seed=7)
    Fo = tlr.factor(tlr.build(x, b, 1e-3, ell, nug, compressor="ara", bs=bs, seed=7), 1e-3, compressor="ara",
                    bs=bs, seed=7, compensation="shift", shift=1e-3)
    Y = inputs.rhs(N, 3, 31)
    Y[:, 2] = 0.0
    Xg, itg, rg = A.pcg(Fm, _t(T, Y), tol=tol, maxit=300)
    Xo, ito, ro = opcg.pcg(lambda Z: tlr.matvec(Ao, Z, "A"), lambda R: tlr.solve(Fo, R), Y, tol, 300)
    Xg = Xg.cpu().numpy()
    assert itg[2] == 0 and ito[2] == 0 and not Xg[:, 2].any()
    for c in range(2):
        assert abs(itg[c] - int(ito[c])) <= 1, (itg, ito)
        assert 0 < itg[c] < 60
        assert rg[c] <= 2 * tol and ro[c] <= 2 * tol
        assert rel(Xg[:, c], Xo[:, c]) < 1e-4
    A.free()
    Fm.free()
