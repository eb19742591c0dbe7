"""Planted mistakes in the oracle (CPU only): each plausible error must fail a pin.

A pin is only worth something if a wrong oracle fails it.  These tests patch
one step of the oracle at a time (dropped term, wrong sign, transposed operand,
off-by-one) and check that the OU closed-form pin or the dense pin rejects it.
"""
import numpy as np
import pytest

import inputs
from oracle import dense, kdtree, kernel, tlr


def _ou_ok(ldl=False):
    try:
        return _ou_check(ldl)
    except dense.NotPositiveDefinite:
        return False


def _ou_check(ldl):
    N, b, ell = 256, 32, 0.3
    x = inputs.points(N, 1, 8)
    A = tlr.build(x, b, 1e-12, ell, 0.0)
    F = tlr.factor(A, 1e-12, ldl=ldl)
    xs = A.xo[:, 0]
    s = np.ones(N)
    s[1:] = np.sqrt(1.0 - np.exp(-2.0 * np.diff(xs) / ell))
    Lex = np.tril(np.exp(-(xs[:, None] - xs[None, :]) / ell) * s[None, :])
    ld = float(np.sum(np.log(1.0 - np.exp(-2.0 * np.diff(xs) / ell))))
    Ld = F.to_dense()
    if ldl:
        Ld = Ld * np.sqrt(np.concatenate(F.d))[None, :]
    return np.allclose(Ld, Lex, atol=1e-8) and abs(tlr.logdet(F) - ld) < 1e-8 * abs(ld)


def _dense_ok():
    try:
        return _dense_check()
    except dense.NotPositiveDefinite:
        return False


def _dense_check():
    x = inputs.points(600, 2, 2)
    A = tlr.build(x, 128, 1e-13, 0.1, 1e-4)
    F = tlr.factor(A, 1e-13)
    Ad = kernel.dense(x, 0.1, 1e-4)
    return np.linalg.norm(tlr.matvec(F, np.eye(600), "LLt") - Ad, 2) < 1e-9 * np.linalg.norm(Ad, 2)


def test_unmutated_oracle_passes():
    assert _ou_ok() and _ou_ok(ldl=True) and _dense_ok()


def test_dropped_term_in_diag_update_is_caught(monkeypatch):
    orig = tlr._diag_update

    def drop_last(F, k):
        D = orig(F, k)
        if k > 0:
            U, V = F.U[(k, k - 1)], F.V[(k, k - 1)]
            D -= U @ (V.T @ V) @ U.T
        return D
    monkeypatch.setattr(tlr, "_diag_update", drop_last)
    assert not _ou_ok()


def test_wrong_sign_in_trsm_is_caught(monkeypatch):
    orig = dense.solve_lower
    monkeypatch.setattr(dense, "solve_lower", lambda L, B, unit=False: -orig(L, B, unit))
    assert not _ou_ok()


def test_transposed_triangular_operand_is_caught(monkeypatch):
    orig = dense.solve_lower
    monkeypatch.setattr(dense, "solve_lower", lambda L, B, unit=False: np.linalg.solve(L.T, B))
    assert not _dense_ok()


def test_missing_D_in_ldl_chain_is_caught(monkeypatch):
    orig = tlr._diag_update

    def no_d(F, k):
        saved = F.d
        F.d = None
        try:
            return orig(F, k)
        finally:
            F.d = saved
    monkeypatch.setattr(tlr, "_diag_update", no_d)
    assert not _ou_ok(ldl=True)


def test_kd_split_off_by_one_is_caught(monkeypatch):
    # the leaf-size rule of Section 6: all leaves hold b points except possibly the last
    x = inputs.points(1000, 2, 3)
    monkeypatch.setattr(kdtree, "_left_size", lambda n, b: n // 2)
    perm = kdtree.kd_order(x, 64)
    monkeypatch.undo()
    assert not np.array_equal(perm, kdtree.kd_order(x, 64))


def test_wrong_sign_in_left_looking_update_is_caught(monkeypatch):
    # Equation 1 with "+" instead of "-": patch the dense form of T through the compressor hook
    orig = tlr._compressor

    def flip(name, eps, bs, seed, stream, k, b):
        c = orig(name, eps, bs, seed, stream, k, b)
        if stream != tlr.STREAM_FACTOR:
            return c
        return lambda T: c(-T)
    monkeypatch.setattr(tlr, "_compressor", flip)
    assert not _ou_ok()


def _schur_mutant(monkeypatch, term):
    from test_oracle_pins import schur_pins_hold
    orig = tlr._schur_compensation

    def mutant(Dk, comp):
        Q, _, _ = comp(Dk)
        Dbar = Q @ (Q.T @ Dk @ Q) @ Q.T
        return term(Dk, Dbar, orig(Dk, comp))

    assert schur_pins_hold()
    monkeypatch.setattr(tlr, "_schur_compensation", mutant)
    return schur_pins_hold()


def test_schur_compensation_by_D_instead_of_its_residual_is_caught(monkeypatch):
    assert not _schur_mutant(monkeypatch, lambda D, Db, ok: np.diag(np.sum(np.abs(D), axis=1)))


def test_schur_compensation_with_wrong_sign_is_caught(monkeypatch):
    assert not _schur_mutant(monkeypatch, lambda D, Db, ok: -ok)


def test_schur_compensation_off_the_diagonal_is_caught(monkeypatch):
    def spread(D, Db, ok):
        r = np.diag(ok)
        return ok + 0.5 * (np.outer(np.sqrt(r), np.sqrt(r)) - np.diag(r))
    assert not _schur_mutant(monkeypatch, spread)


def _pivot_mutant(monkeypatch, name, fn):
    from test_oracle_pins import pivoted_pins_hold
    assert pivoted_pins_hold()
    monkeypatch.setattr(tlr, name, fn)
    return pivoted_pins_hold()


def test_pivot_by_smallest_tile_is_caught(monkeypatch):
    def smallest(Ad, D, k):
        return k + int(np.argmin([np.linalg.norm(Ad[i] - D[i]) for i in range(k, len(Ad))]))
    assert not _pivot_mutant(monkeypatch, "_select_pivot", smallest)


def test_pivot_without_exchanging_factored_rows_is_caught(monkeypatch):
    orig = tlr._swap_tiles

    def keep_rows(F, Ad, At, k, p):
        saved = {j: (F.U[(k, j)], F.V[(k, j)], F.U[(p, j)], F.V[(p, j)]) for j in range(k)}
        out = orig(F, Ad, At, k, p)
        for j, (uk, vk, up, vp) in saved.items():
            F.U[(k, j)], F.V[(k, j)], F.U[(p, j)], F.V[(p, j)] = uk, vk, up, vp
        return out
    assert not _pivot_mutant(monkeypatch, "_swap_tiles", keep_rows)


def test_pivot_without_transposing_crossing_tiles_is_caught(monkeypatch):
    def no_transpose(F, Ad, At, k, p):
        sig = lambda i: p if i == k else (k if i == p else i)
        Ad[k], Ad[p] = Ad[p], Ad[k]
        for j in range(k):
            F.U[(k, j)], F.U[(p, j)] = F.U[(p, j)], F.U[(k, j)]
            F.V[(k, j)], F.V[(p, j)] = F.V[(p, j)], F.V[(k, j)]
        return {(i, j): (At[(sig(i), sig(j))] if sig(i) > sig(j) else At[(sig(j), sig(i))]) for (i, j) in At}
    assert not _pivot_mutant(monkeypatch, "_swap_tiles", no_transpose)


def test_modified_cholesky_shifting_instead_of_clamping_is_caught(monkeypatch):
    """A plausible variant adds delta to every block eigenvalue instead of raising only those below it."""
    from test_oracle_pins import test_modified_cholesky_closed_forms
    test_modified_cholesky_closed_forms()
    monkeypatch.setattr(dense, "_modify_eigenvalues", lambda w, d: w + d)
    with pytest.raises((AssertionError, dense.NotPositiveDefinite)):
        test_modified_cholesky_closed_forms()


def test_update_sum_pairing_the_wrong_columns_is_caught(monkeypatch):
    """Equation 1's sum as one product of concatenated factors: the right-hand blocks must pair with
    the left-hand blocks of the same column j.  Reversing their order pairs j with k-1-j.  (The 1D
    closed form cannot see this: there every U_ij of a block row spans the same direction.)"""
    def misaligned(F, i, l, k):
        if k == 0:
            return np.zeros((F.b, F.b))
        left = np.hstack([F.U[(i, j)] @ (F.V[(i, j)].T @ tlr._dv(F, j, F.V[(l, j)])) for j in range(k)])
        right = np.hstack([F.U[(l, j)] for j in reversed(range(k))])
        return left @ right.T
    monkeypatch.setattr(tlr, "_update_sum", misaligned)
    assert not _dense_ok()


def test_update_sum_stopping_one_column_early_is_caught(monkeypatch):
    orig = tlr._update_sum
    monkeypatch.setattr(tlr, "_update_sum", lambda F, i, l, k: orig(F, i, l, max(k - 1, 0)))
    assert not _ou_ok() and not _ou_ok(ldl=True)


# ---------------------------------------------------------------- rank trimming (Section 6)
def _trim_variant(keep, scale=True, transpose=True):
    def trim(Q, B, eps):
        W, sv, Zt = np.linalg.svd(B, full_matrices=False)
        r = keep(sv, eps)
        Z = Zt[:r].T if transpose else Zt[:, :r]
        return Q @ Z, (W[:, :r] * sv[:r]) if scale else W[:, :r]
    return trim


def test_unmutated_trim_variant_passes():
    from test_oracle_pins import trim_pins_hold
    assert trim_pins_hold(_trim_variant(lambda sv, eps: int(np.count_nonzero(sv > eps))))


@pytest.mark.parametrize("name,variant", [
    ("keeps the values below eps", _trim_variant(lambda sv, eps: int(np.count_nonzero(sv < eps)))),
    ("drops one value too many", _trim_variant(lambda sv, eps: int(np.count_nonzero(sv > eps)) - 1)),
    ("keeps one value too many", _trim_variant(lambda sv, eps: int(np.count_nonzero(sv > eps)) + 1)),
    ("forgets the singular values", _trim_variant(lambda sv, eps: int(np.count_nonzero(sv > eps)), scale=False)),
    ("takes Z's rows for its columns", _trim_variant(lambda sv, eps: int(np.count_nonzero(sv > eps)), transpose=False)),
])
def test_trim_mistakes_are_caught(name, variant):
    from test_oracle_pins import trim_pins_hold
    assert not trim_pins_hold(variant), name
