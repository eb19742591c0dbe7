"""The allocation-free kernel-matrix product (tlr_kernel_matvec_noalloc).

Callers that cannot allocate device memory (a memory manager owns the device
heap, or cudaMalloc's synchronization is not acceptable) use this entry point:
it stages the points in a fixed device array inside the library instead of
allocating.  Its results must equal those of the allocating entry point
tlr_kernel_matvec, including when two calls in a row reuse the shared array.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def _noalloc(T):
    f = C.CDLL(T.library_path()).tlr_kernel_matvec_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.POINTER(T.Kernel), C.c_int, C.c_void_p, C.c_int64,
                  C.c_void_p, C.c_int64]
    return f


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch

    import paper_2108_11932_gb300 as T
    T.build()
    f = _noalloc(T)
    ctx = T.Context(0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for N, d, nrhs, ell, nug, seed in [(3000, 3, 5, 0.2, 1e-4, 1), (2048, 2, 2, 0.1, 1e-4, 2)]:
        x = inputs.points(N, d, seed)
        Z = T.fortran(torch.tensor(inputs.rhs(N, nrhs, seed), device="cuda:0"))
        Y = T.fortran(torch.full((N, nrhs), np.nan, dtype=torch.float64, device="cuda:0"))
        k = T.Kernel(0, ell, nug)
        st = f(stream, x.ctypes.data, N, d, C.byref(k), nrhs, Z.data_ptr(), N, Y.data_ptr(), N)
        assert st == T.OK
        torch.cuda.synchronize()
        ref = ctx.kernel_matvec(x, ell, nug, Z)
        err = float((Y - ref).abs().max() / ref.abs().max())
        assert err <= 1e-13, err


def test_noalloc_rejects_sizes_above_its_array():
    import paper_2108_11932_gb300 as T
    T.build()
    f = _noalloc(T)
    x = np.zeros((4, 3))
    k = T.Kernel(0, 0.1, 1e-4)
    # N * d beyond the fixed array: rejected before any pointer is read
    assert f(None, x.ctypes.data, 131073, 3, C.byref(k), 1, 1, 131073, 1, 131073) == T.ERR_LIMIT
    assert f(None, x.ctypes.data, 4, 3, C.byref(k), 1, None, 4, None, 4) == T.ERR_ARG
