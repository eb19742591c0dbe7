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
