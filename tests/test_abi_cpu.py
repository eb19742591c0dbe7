"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol declared in include/tlr.h, and its host-side KD ordering matches the
oracle's bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

import inputs
from oracle import kdtree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2108_11932_gb300 as T
    T.build()
    return T


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "tlr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(tlr_[a-z0-9_]+)\s*\(", txt))
    types = set(re.findall(r"typedef\s+[^;]*?\(\s*\*\s*(tlr_[a-z0-9_]+)\s*\)", txt))
    return sorted(names - types)


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for s in ["tlr_compress", "tlr_potrf", "tlr_ldlt", "tlr_solve", "tlr_logdet", "tlr_matvec", "tlr_create"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.library_path())
    missing = [s for s in _declared_symbols() if not hasattr(so, s)]
    assert not missing, missing


def test_opts_default_and_strerror(lib):
    o = lib.default_opts()
    assert o.bs == 16 and o.precision == 0 and o.compensation == 0 and o.max_slots == 0
    so = lib._load()
    assert so.tlr_strerror(-3).decode().startswith("matrix not positive definite")


def test_null_arguments_are_rejected_without_gpu(lib):
    so = lib._load()
    assert so.tlr_compress(None, None, 0, 2, None, 0, 0.0, None, None) == lib.ERR_ARG
    assert so.tlr_potrf(None, None, 1e-6, None) == lib.ERR_ARG
    assert so.tlr_destroy(None) == lib.ERR_ARG
    assert so.tlr_solve(None, None, 1, None, 1) == lib.ERR_ARG
    it = (ctypes.c_int * 1)()
    rr = (ctypes.c_double * 1)()
    assert so.tlr_pcg(None, None, None, 1, None, 1, None, 1, 1e-6, 10, it, rr) == lib.ERR_ARG
    assert so.tlr_trim(None, None, 1e-6) == lib.ERR_ARG
    assert so.tlr_trim_tiles(None, 1, 16, 4, None, None, 1e-6, None, None, None) == lib.ERR_ARG


@pytest.mark.parametrize("N,d,b,seed", [(4096, 2, 256, 0), (5000, 3, 512, 1), (1000, 1, 64, 3), (777, 2, 100, 4),
                                        (50, 2, 64, 5), (32768, 3, 512, 1)])
def test_kd_order_bit_exact_vs_oracle(lib, N, d, b, seed):
    x = inputs.points(N, d, seed)
    assert np.array_equal(lib.kd_order(x, b), kdtree.kd_order(x, b))


def test_autotune_choose_takes_the_nearest_class_of_the_same_dimension():
    from paper_2108_11932_gb300 import autotune
    table = {(2, 11): (128, 16, 0), (2, 14): (256, 32, 16), (3, 12): (256, 16, 0)}
    assert autotune.choose(table, 2048, 2) == (128, 16, 0)
    assert autotune.choose(table, 3000, 2) == (128, 16, 0)     # bucket 12: 11 and 14 -> nearer 11
    assert autotune.choose(table, 12000, 2) == (256, 32, 16)   # bucket 14
    assert autotune.choose(table, 65536, 3) == (256, 16, 0)
    assert autotune.choose(table, 4096, 1) == autotune.DEFAULT  # no class of that dimension


def test_kernel_products_share_their_argument_rule(lib):
    """tlr_kernel_matvec and tlr_kernel_matvec_noalloc compute the same Y = A X and reject the same
    arguments before touching the GPU: an unknown kernel type and a nugget of -1 (a zero diagonal) among them."""
    so = lib._load()
    so.tlr_kernel_matvec_noalloc.restype = ctypes.c_int
    pts = np.zeros((4, 2))
    X = (ctypes.c_double * 4)()
    Y = (ctypes.c_double * 4)()
    dummy_ctx = ctypes.create_string_buffer(4096)  # never dereferenced: the arguments are rejected first
    for ktype, ell, nug in [(7, 0.1, 0.0), (0, 0.1, -1.0), (0, 0.1, -2.5), (0, 0.0, 0.0), (0, -0.1, 0.0)]:
        k = lib.Kernel(ktype, ell, nug)
        a = so.tlr_kernel_matvec(ctypes.cast(dummy_ctx, ctypes.c_void_p), pts.ctypes.data, 4, 2, ctypes.byref(k), 1,
                                 ctypes.cast(X, ctypes.c_void_p), 4, ctypes.cast(Y, ctypes.c_void_p), 4)
        b = so.tlr_kernel_matvec_noalloc(None, ctypes.c_void_p(pts.ctypes.data), ctypes.c_int64(4), 2, ctypes.byref(k),
                                         1, ctypes.cast(X, ctypes.c_void_p), ctypes.c_int64(4),
                                         ctypes.cast(Y, ctypes.c_void_p), ctypes.c_int64(4))
        assert a == b == lib.ERR_ARG, (ktype, ell, nug, a, b)


def test_submit_rejects_bad_requests_without_gpu(lib):
    """tlr_submit validates a request before it touches the context or the GPU."""
    so = lib._load()
    pts = np.zeros((8, 2))
    dummy_ctx = ctypes.create_string_buffer(8192)  # never dereferenced for a rejected request
    t = ctypes.c_uint64(0)

    def req(**kw):
        r = lib.Request(pts.ctypes.data, 8, 2, lib.Kernel(0, 0.1, 1e-4), 4, 1e-6, 0, 0, None, lib.default_opts(bs=4))
        for k, v in kw.items():
            setattr(r, k, v)
        return r
    bad = [req(N=0), req(d=4), req(eps=0.0), req(b=0), req(nrhs=2), req(ldl=2), req(kernel=lib.Kernel(1, 0.1, 0.0)),
           req(kernel=lib.Kernel(0, 0.1, -1.0)), req(opts=lib.default_opts(bs=8)), req(points=None),
           # tile pivoting (Algorithm 9): Cholesky only, FP64, no padded tile (N a multiple of b)
           req(opts=lib.default_opts(bs=4, pivot=lib.PIVOT_FROBENIUS), ldl=1),
           req(opts=lib.default_opts(bs=4, pivot=lib.PIVOT_FROBENIUS), N=7),
           req(opts=lib.default_opts(bs=4, pivot=lib.PIVOT_FROBENIUS, precision=lib.PREC_MIXED)),
           req(opts=lib.default_opts(bs=4, pivot=lib.PIVOT_FROBENIUS, compensation=lib.COMP_SCHUR)),
           req(opts=lib.default_opts(bs=4, pivot=2))]
    for r in bad:
        assert so.tlr_submit(ctypes.cast(dummy_ctx, ctypes.c_void_p), ctypes.byref(r), ctypes.byref(t)) == lib.ERR_ARG
    assert so.tlr_submit(None, ctypes.byref(req()), ctypes.byref(t)) == lib.ERR_ARG
    assert so.tlr_progress(None, None, None) == lib.ERR_ARG
    res = lib.Result()
    assert so.tlr_poll(None, 1, ctypes.byref(res), None, 1) == lib.ERR_ARG
