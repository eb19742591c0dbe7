"""Exact kernel product in plain C (oracle; test infrastructure).

`kernel_matvec.c` generates A_ij = exp(-||x_i - x_j||_2 / ell) + nugget * delta_ij (Section 6)
entry by entry and multiplies, with OpenMP threads over rows: the same product as
`kernel.matvec`, fast enough for the power iterations of Section 6's accuracy check at
N = 131072.  It is compiled on first use with the host C compiler into `oracle/_build/`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kernel_matvec.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_kernel_matvec.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C source (plain gcc -O2 -fopenmp, no machine-specific flags); returns the path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_kernel_matvec.restype = ctypes.c_int
        lib.oracle_kernel_matvec.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the product uses."""
    return int(_load().oracle_num_threads())


def matvec(xo: np.ndarray, ell: float, nugget: float, X: np.ndarray) -> np.ndarray:
    """A @ X for the kernel matrix of the points xo (N x d); X is N or N x nrhs (nrhs <= 64)."""
    xo = np.ascontiguousarray(xo, dtype=np.float64)
    N, d = xo.shape
    vec = np.ndim(X) == 1
    Xf = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(N, -1))
    Y = np.zeros_like(Xf, order="F")
    st = _load().oracle_kernel_matvec(xo.ctypes.data, N, d, float(ell), float(nugget), Xf.shape[1],
                                      Xf.ctypes.data, Y.ctypes.data)
    if st != 0:
        raise ValueError("kernel_matvec: unsupported arguments")
    return Y[:, 0] if vec else Y
