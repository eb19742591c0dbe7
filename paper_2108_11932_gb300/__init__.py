"""GB300 tile-low-rank (TLR) Cholesky / LDL^T: thin Python binding of libtlr_gb300.so.

Argument marshalling only: every step of the factorization runs in the CUDA
library through its C ABI (include/tlr.h).  PyTorch provides device memory
(its caching allocator, passed to the library as allocation callbacks) and the
CUDA stream.  If the library is not built, importing the binding's entry points
raises: there is no CPU fallback.

Matrices handed to the library are column-major: a torch tensor of shape
(rows, cols) with stride (1, rows) (see `fortran`).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build  # noqa: F401

__all__ = ["Context", "Matrix", "Opts", "TLRError", "build", "fortran", "kd_order", "library_path"]

OK, ERR_ARG, ERR_NOMEM, ERR_NOT_SPD, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_LIMIT = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP64, PREC_FP32, PREC_MIXED = 0, 1, 2
COMP_NONE, COMP_SHIFT, COMP_SCHUR, COMP_MODCHOL = 0, 1, 2, 3
PIVOT_NONE, PIVOT_FROBENIUS = 0, 1
OP_A, OP_L, OP_LT, OP_LLT = 0, 1, 2, 3
STREAM_COMPRESS, STREAM_FACTOR, STREAM_SCHUR = 1, 2, 3


class TLRError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_strerror(status)} ({status})")
        self.status = status


class Opts(C.Structure):
    _fields_ = [("bs", C.c_int), ("max_slots", C.c_int), ("precision", C.c_int), ("compensation", C.c_int),
                ("shift", C.c_double), ("seed", C.c_uint64), ("ldl", C.c_int), ("pivot", C.c_int),
                ("reserved", C.c_int * 6)]


class Kernel(C.Structure):
    _fields_ = [("type", C.c_int), ("ell", C.c_double), ("nugget", C.c_double)]


class Info(C.Structure):
    _fields_ = [("N", C.c_int64), ("b", C.c_int), ("nb", C.c_int), ("d", C.c_int), ("state", C.c_int),
                ("k_fail", C.c_int), ("max_rank", C.c_int), ("mean_rank", C.c_double), ("bytes", C.c_int64),
                ("flops_exec", C.c_double), ("flops_model", C.c_double), ("ara_rounds", C.c_double),
                ("seconds", C.c_double), ("flops_fp32", C.c_double), ("tile_rounds_fp32", C.c_double),
                ("tile_rounds_fp64", C.c_double)]


class Request(C.Structure):
    _fields_ = [("points", C.c_void_p), ("N", C.c_int64), ("d", C.c_int), ("kernel", Kernel), ("b", C.c_int),
                ("eps", C.c_double), ("ldl", C.c_int), ("nrhs", C.c_int), ("rhs", C.c_void_p), ("opts", Opts)]


class Result(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("retried", C.c_int), ("sign", C.c_int),
                ("logdet", C.c_double), ("wait_s", C.c_double), ("run_s", C.c_double), ("bytes", C.c_int64),
                ("mean_rank", C.c_double)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_lib = None
P = C.c_void_p
D = C.POINTER(C.c_double)


def library_path() -> str:
    return LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"{LIB} is not built: call paper_2108_11932_gb300.build() first")
    L = C.CDLL(LIB)
    sig = {
        "tlr_opts_default": (None, [C.POINTER(Opts)]),
        "tlr_strerror": (C.c_char_p, [C.c_int]),
        "tlr_create": (C.c_int, [C.POINTER(P), C.c_int, C.c_size_t, P, _ALLOC, _FREE, P]),
        "tlr_destroy": (C.c_int, [P]),
        "tlr_compress": (C.c_int, [P, P, C.c_int64, C.c_int, C.POINTER(Kernel), C.c_int, C.c_double,
                                   C.POINTER(Opts), C.POINTER(P)]),
        "tlr_copy": (C.c_int, [P, P, C.POINTER(P)]),
        "tlr_compress_ordered": (C.c_int, [P, P, P, C.c_int64, C.c_int, C.POINTER(Kernel), C.c_int, C.c_double,
                                           C.POINTER(Opts), C.POINTER(P)]),
        "tlr_gemm_stats": (C.c_int, [P, C.c_int, D, D, D, C.POINTER(C.c_int64)]),
        "tlr_factor_batch": (C.c_int, [P, C.c_int, C.POINTER(P), D, C.POINTER(Opts), C.c_int, C.POINTER(C.c_int)]),
        "tlr_session_create": (C.c_int, [P, C.POINTER(P)]),
        "tlr_session_destroy": (C.c_int, [P]),
        "tlr_session_add": (C.c_int, [P, P, C.c_double, C.POINTER(Opts), C.c_int, C.POINTER(C.c_int)]),
        "tlr_session_step": (C.c_int, [P, C.POINTER(C.c_int)]),
        "tlr_session_poll": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "tlr_potrf": (C.c_int, [P, P, C.c_double, C.POINTER(Opts)]),
        "tlr_ldlt": (C.c_int, [P, P, C.c_double, C.POINTER(Opts)]),
        "tlr_solve": (C.c_int, [P, P, C.c_int, P, C.c_int64]),
        "tlr_logdet": (C.c_int, [P, P, D, C.POINTER(C.c_int)]),
        "tlr_pcg": (C.c_int, [P, P, P, C.c_int, P, C.c_int64, P, C.c_int64, C.c_double, C.c_int,
                              C.POINTER(C.c_int), D]),
        "tlr_matvec": (C.c_int, [P, P, C.c_int, C.c_int, P, C.c_int64, P, C.c_int64]),
        "tlr_kernel_matvec": (C.c_int, [P, P, C.c_int64, C.c_int, C.POINTER(Kernel), C.c_int, P, C.c_int64, P,
                                        C.c_int64]),
        "tlr_get_info": (C.c_int, [P, C.POINTER(Info)]),
        "tlr_get_ranks": (C.c_int, [P, P, P]),
        "tlr_get_perm": (C.c_int, [P, P]),
        "tlr_get_tile": (C.c_int, [P, P, C.c_int, C.c_int, P, P]),
        "tlr_free": (C.c_int, [P, P]),
        "tlr_kd_order": (C.c_int, [P, C.c_int64, C.c_int, C.c_int, P]),
        "tlr_omega": (C.c_int, [P, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_int, P]),
        "tlr_ara_dense": (C.c_int, [P, C.c_int, C.c_int, P, C.c_int, C.c_double, C.c_uint64, C.c_uint32,
                                    C.c_uint32, P, P, P]),
        "tlr_dense_potrf": (C.c_int, [P, C.c_int, P, C.c_int, C.POINTER(C.c_int)]),
        "tlr_trim_tiles": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, C.c_double, P, P, P]),
        "tlr_trim": (C.c_int, [P, P, C.c_double]),
        "tlr_dense_modchol": (C.c_int, [P, C.c_int, P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "tlr_dense_ldlt": (C.c_int, [P, C.c_int, P, C.c_int, C.POINTER(C.c_int)]),
        "tlr_dense_trsm": (C.c_int, [P, C.c_int, P, C.c_int, C.c_int, C.c_int, P, C.c_int]),
        "tlr_split_product": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P, C.c_int, P, C.c_int]),
        "tlr_fp64_peak": (C.c_int, [P, D]),
        "tlr_submit": (C.c_int, [P, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "tlr_progress": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "tlr_poll": (C.c_int, [P, C.c_uint64, C.POINTER(Result), P, C.c_int64]),
        "tlr_split_planes": (C.c_int, [P, C.POINTER(C.c_int64), D, C.c_int]),
        "tlr_launch_count": (C.c_int64, [P]),
        "tlr_profile": (C.c_int, [P, C.c_int, D, C.POINTER(C.c_int64), C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _strerror(s: int) -> str:
    try:
        return _load().tlr_strerror(s).decode()
    except Exception:
        return "unknown"


def _check(st: int, what: str):
    if st != OK:
        raise TLRError(st, what)


def _ptr(t) -> int:
    return t.data_ptr()


def fortran(x):
    """Column-major copy of a 2D torch tensor (shape kept, stride (1, rows))."""
    return x.t().contiguous().t()


def _ld(t) -> int:
    if t.dim() == 1 or t.shape[1] == 1:
        return max(t.shape[0], 1)
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError("matrices must be column-major: use fortran(x)")
    return max(t.stride(1), t.shape[0], 1)


def default_opts(**kw) -> Opts:
    o = Opts()
    _load().tlr_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def kd_order(points: np.ndarray, b: int) -> np.ndarray:
    """KD-tree permutation of Section 6 (library host code)."""
    x = np.ascontiguousarray(points, dtype=np.float64)
    N, d = x.shape
    perm = np.empty(N, dtype=np.int64)
    _check(_load().tlr_kd_order(x.ctypes.data, N, d, b, perm.ctypes.data), "tlr_kd_order")
    return perm


class Context:
    """A library context bound to one GPU and one CUDA stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = True, hbm_budget: int = 0):
        import torch
        L = _load()
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._cbs = None
        alloc, free = _ALLOC(), _FREE()
        if torch_allocator:
            cuda_stream = self.stream.cuda_stream

            def _a(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, cuda_stream)
                except Exception:
                    return None

            def _f(p, user):
                torch.cuda.caching_allocator_delete(p)
            alloc, free = _ALLOC(_a), _FREE(_f)
            self._cbs = (alloc, free)
        h = P()
        _check(L.tlr_create(C.byref(h), device, int(hbm_budget), P(self.stream.cuda_stream), alloc, free, None),
               "tlr_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _check(_load().tlr_destroy(self.h), "tlr_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launches(self) -> int:
        return int(_load().tlr_launch_count(self.h))

    # ---- TLR construction
    def compress(self, points: np.ndarray, b: int, eps: float, ell: float, nugget: float, opts: Opts | None = None):
        x = np.ascontiguousarray(points, dtype=np.float64)
        N, d = x.shape
        k = Kernel(0, ell, nugget)
        m = P()
        _check(_load().tlr_compress(self.h, x.ctypes.data, N, d, C.byref(k), b, eps,
                                    C.byref(opts) if opts else None, C.byref(m)), "tlr_compress")
        return Matrix(self, m)

    def compress_ordered(self, pts, perm: np.ndarray | None, b: int, eps: float, ell: float, nugget: float,
                         opts: Opts | None = None):
        """Construction from device points already in KD order (pts: (N, d) contiguous float64 cuda tensor)."""
        if not pts.is_contiguous():
            raise ValueError("pts must be a contiguous (N, d) tensor")
        N, d = pts.shape
        pp = None
        if perm is not None:
            pp = np.ascontiguousarray(perm, dtype=np.int64)
        k = Kernel(0, ell, nugget)
        m = P()
        _check(_load().tlr_compress_ordered(self.h, _ptr(pts), pp.ctypes.data if pp is not None else None, N, d,
                                            C.byref(k), b, eps, C.byref(opts) if opts else None, C.byref(m)),
               "tlr_compress_ordered")
        return Matrix(self, m)

    def factor_batch(self, mats: list, eps, opts=None, ldl: bool = False) -> list:
        """Factor several matrices together (one dynamic batch per column step); returns statuses."""
        n = len(mats)
        hs = (P * n)(*[m.h for m in mats])
        ev = (C.c_double * n)(*([eps] * n if np.isscalar(eps) else list(eps)))
        if opts is None:
            op = None
        else:
            ol = [opts] * n if isinstance(opts, Opts) else list(opts)
            op = (Opts * n)(*ol)
        st = (C.c_int * n)()
        _check(_load().tlr_factor_batch(self.h, n, hs, ev, op, int(ldl), st), "tlr_factor_batch")
        return [st[i] for i in range(n)]

    GEMM_FAMILIES = ["fp64_NN", "fp64_TN", "fp64_NT", "fp32_NN", "fp32_TN", "fp32_NT", "split_planes", "orth_fp64"]

    def gemm_stats(self, enable: bool = True) -> dict:
        """Return (and reset) per-family GEMM launch accounting; switch it on/off."""
        nf = len(self.GEMM_FAMILIES)
        ms = (C.c_double * nf)()
        fl = (C.c_double * nf)()
        by = (C.c_double * nf)()
        ln = (C.c_int64 * nf)()
        _check(_load().tlr_gemm_stats(self.h, int(enable), ms, fl, by, ln), "tlr_gemm_stats")
        return {f: {"ms": ms[i], "flops": fl[i], "bytes": by[i], "launches": ln[i]}
                for i, f in enumerate(self.GEMM_FAMILIES)}

    def kernel_matvec(self, points: np.ndarray, ell: float, nugget: float, X):
        x = np.ascontiguousarray(points, dtype=np.float64)
        N, d = x.shape
        X2 = X if X.dim() == 2 else X[:, None]
        Y = self.torch.empty_like(X2)
        Y = fortran(Y)
        k = Kernel(0, ell, nugget)
        _check(_load().tlr_kernel_matvec(self.h, x.ctypes.data, N, d, C.byref(k), X2.shape[1], _ptr(X2), _ld(X2),
                                         _ptr(Y), _ld(Y)), "tlr_kernel_matvec")
        return Y if X.dim() == 2 else Y[:, 0]

    # ---- building blocks
    def omega(self, seed: int, stream: int, k: int, t: int, b: int, bs: int):
        out = self.torch.empty((bs, b), dtype=self.torch.float64, device=f"cuda:{self.device}").t()
        _check(_load().tlr_omega(self.h, seed, stream, k, t, b, bs, _ptr(out)), "tlr_omega")
        return out

    def ara_dense(self, T, bs: int, eps: float, seed: int, stream: int = STREAM_COMPRESS, k: int = 0):
        """T: (nops, n, n) tensor whose [s] slices are column-major operands (T[s].t() row-major)."""
        torch = self.torch
        nops, n, _ = T.shape
        Tc = T.contiguous()
        Q = torch.zeros_like(Tc)
        B = torch.zeros_like(Tc)
        r = torch.zeros(nops, dtype=torch.int32, device=Tc.device)
        _check(_load().tlr_ara_dense(self.h, nops, n, _ptr(Tc), bs, eps, seed, stream, k, _ptr(Q), _ptr(B), _ptr(r)),
               "tlr_ara_dense")
        return Q, B, r

    def trim_tiles(self, Q, B, eps: float):
        """ARA -> SVD rank trimming of tiles Q[t] B[t]^T: Q, B (ntiles, r, b) tensors whose [t] slices are
        column-major b x r blocks.  Returns (Q', B', ranks) with the first ranks[t] columns kept."""
        torch = self.torch
        nt, r, b = Q.shape
        Qc, Bc = Q.contiguous(), B.contiguous()
        Qo, Bo = torch.empty_like(Qc), torch.empty_like(Bc)
        rk = np.zeros(nt, dtype=np.int32)
        _check(_load().tlr_trim_tiles(self.h, nt, b, r, _ptr(Qc), _ptr(Bc), eps, _ptr(Qo), _ptr(Bo),
                                      rk.ctypes.data), "tlr_trim_tiles")
        return Qo, Bo, rk

    def dense_modchol(self, A):
        """Modified Cholesky (Algorithm 8) in place; returns (modified, info)."""
        mod, info = C.c_int(0), C.c_int(0)
        _check(_load().tlr_dense_modchol(self.h, A.shape[0], _ptr(A), _ld(A), C.byref(mod), C.byref(info)),
               "tlr_dense_modchol")
        return mod.value, info.value

    def dense_potrf(self, A, ldl: bool = False):
        info = C.c_int(0)
        f = _load().tlr_dense_ldlt if ldl else _load().tlr_dense_potrf
        _check(f(self.h, A.shape[0], _ptr(A), _ld(A), C.byref(info)), "tlr_dense_potrf")
        return info.value

    def dense_trsm(self, L, B, unit: bool = False):
        _check(_load().tlr_dense_trsm(self.h, L.shape[0], _ptr(L), _ld(L), int(unit), B.shape[1], _ptr(B), _ld(B)),
               "tlr_dense_trsm")

    def split_product(self, T, X, trans=False, out=None):
        """C = T X (trans False/0, or 2: A read by columns) or T^T X (True/1) on the tcgen05 tensor cores by exact
        splitting into 7-bit chunk planes."""
        n, ncols = T.shape[0], X.shape[1]
        C_ = out if out is not None else fortran(self.torch.empty((n, ncols), dtype=self.torch.float64,
                                                                   device=T.device))
        _check(_load().tlr_split_product(self.h, int(trans), n, ncols, _ptr(T), _ptr(X), _ld(X), _ptr(C_), _ld(C_)),
               "tlr_split_product")
        return C_

    PHASES = ["gram", "diag_update", "potrf", "sample", "orthog", "host_sync", "project", "trsm", "update_tiles",
              "compress", "solve", "other", "host_blocked"]

    def profile(self, enable: bool = True) -> dict:
        """Return (and reset) the phase profile {phase: (ms, launches)}; switch profiling on/off."""
        n = len(self.PHASES)
        ms = (C.c_double * n)()
        ln = (C.c_int64 * n)()
        _check(_load().tlr_profile(self.h, int(enable), ms, ln, n), "tlr_profile")
        return {p: (ms[i], ln[i]) for i, p in enumerate(self.PHASES)}

    def split_planes(self, reset: bool = True) -> tuple[list, float]:
        """Output blocks of the split products by 7-bit planes used (index 1..8) and chunk bytes read."""
        c = (C.c_int64 * 9)()
        by = C.c_double(0)
        _check(_load().tlr_split_planes(self.h, c, C.byref(by), int(reset)), "tlr_split_planes")
        return [c[i] for i in range(9)], by.value

    # ---- serving queue (tlr_submit / tlr_progress / tlr_poll)
    def submit(self, points: np.ndarray, b: int, eps: float, ell: float, nugget: float, rhs: np.ndarray | None = None,
               opts: Opts | None = None, ldl: bool = False) -> int:
        """Queue one factor + solve + logdet request; the library copies points and rhs."""
        x = np.ascontiguousarray(points, dtype=np.float64)
        N, d = x.shape
        r = None if rhs is None else np.asfortranarray(np.asarray(rhs, dtype=np.float64).reshape(N, -1))
        rq = Request(x.ctypes.data, N, d, Kernel(0, ell, nugget), b, eps, int(ldl), 0 if r is None else r.shape[1],
                     None if r is None else r.ctypes.data, opts if opts is not None else default_opts())
        t = C.c_uint64(0)
        _check(_load().tlr_submit(self.h, C.byref(rq), C.byref(t)), "tlr_submit")
        return t.value

    def progress(self) -> tuple[int, int]:
        """One scheduling step (admission, one column step, finished requests); (queued, in flight)."""
        q, f = C.c_int(0), C.c_int(0)
        _check(_load().tlr_progress(self.h, C.byref(q), C.byref(f)), "tlr_progress")
        return q.value, f.value

    def poll(self, ticket: int, N: int = 0, nrhs: int = 0):
        """None while the request runs; else (result dict, solution N x nrhs or None).  A finished
        request is released by the poll that returns it."""
        res = Result()
        X = np.zeros((N, nrhs), order="F") if N and nrhs else None
        _check(_load().tlr_poll(self.h, ticket, C.byref(res), X.ctypes.data if X is not None else None, max(N, 1)),
               "tlr_poll")
        if not res.done:
            return None
        return {f: getattr(res, f) for f, _ in Result._fields_}, X

    def fp64_peak(self) -> float:
        v = C.c_double(0)
        _check(_load().tlr_fp64_peak(self.h, C.byref(v)), "tlr_fp64_peak")
        return v.value


class Session:
    """Factorizations in flight (continuous batching): add() between step() calls."""

    def __init__(self, ctx: "Context"):
        self.ctx = ctx
        h = P()
        _check(_load().tlr_session_create(ctx.h, C.byref(h)), "tlr_session_create")
        self.h = h
        self.mats = {}

    def add(self, A: "Matrix", eps: float, opts: Opts | None = None, ldl: bool = False) -> int:
        t = C.c_int(0)
        _check(_load().tlr_session_add(self.h, A.h, eps, C.byref(opts) if opts else None, int(ldl), C.byref(t)),
               "tlr_session_add")
        self.mats[t.value] = A
        return t.value

    def step(self) -> int:
        n = C.c_int(0)
        _check(_load().tlr_session_step(self.h, C.byref(n)), "tlr_session_step")
        return n.value

    def poll(self, ticket: int) -> tuple[bool, int]:
        f, st = C.c_int(0), C.c_int(0)
        _check(_load().tlr_session_poll(self.h, ticket, C.byref(f), C.byref(st)), "tlr_session_poll")
        return bool(f.value), st.value

    def close(self):
        if getattr(self, "h", None):
            _load().tlr_session_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """A device-resident TLR matrix or factor (owns a tlr_mat*)."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    def free(self):
        if getattr(self, "h", None) and self.ctx.h:
            _load().tlr_free(self.ctx.h, self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def copy(self) -> "Matrix":
        m = P()
        _check(_load().tlr_copy(self.ctx.h, self.h, C.byref(m)), "tlr_copy")
        return Matrix(self.ctx, m)

    def potrf(self, eps: float, opts: Opts | None = None):
        _check(_load().tlr_potrf(self.ctx.h, self.h, eps, C.byref(opts) if opts else None), "tlr_potrf")
        return self

    def trim(self, eps: float):
        """ARA -> SVD rank trimming of every off-diagonal tile (in place; ranks never grow)."""
        _check(_load().tlr_trim(self.ctx.h, self.h, eps), "tlr_trim")
        return self

    def ldlt(self, eps: float, opts: Opts | None = None):
        _check(_load().tlr_ldlt(self.ctx.h, self.h, eps, C.byref(opts) if opts else None), "tlr_ldlt")
        return self

    def solve(self, B):
        """In place: B (N x nrhs column-major device tensor, original order) <- F^{-1} B."""
        B2 = B if B.dim() == 2 else B[:, None]
        _check(_load().tlr_solve(self.ctx.h, self.h, B2.shape[1], _ptr(B2), _ld(B2)), "tlr_solve")
        return B

    def pcg(self, F: "Matrix", B, tol: float = 1e-6, maxit: int = 300):
        """PCG on this compressed matrix (the operator) with the factor F as preconditioner.

        Returns (X, iterations per column, true relative residual per column); B is not modified."""
        B2 = B if B.dim() == 2 else B[:, None]
        X = fortran(self.ctx.torch.empty_like(B2))
        k = B2.shape[1]
        it = (C.c_int * max(k, 1))()
        rr = (C.c_double * max(k, 1))()
        _check(_load().tlr_pcg(self.ctx.h, self.h, F.h, k, _ptr(B2), _ld(B2), _ptr(X), _ld(X), float(tol), int(maxit),
                               it, rr), "tlr_pcg")
        return X, [it[c] for c in range(k)], [rr[c] for c in range(k)]

    def logdet(self) -> tuple[float, int]:
        v, s = C.c_double(0), C.c_int(0)
        _check(_load().tlr_logdet(self.ctx.h, self.h, C.byref(v), C.byref(s)), "tlr_logdet")
        return v.value, s.value

    def matvec(self, X, op: int = OP_LLT):
        X2 = X if X.dim() == 2 else X[:, None]
        Y = fortran(self.ctx.torch.empty_like(X2))
        _check(_load().tlr_matvec(self.ctx.h, self.h, op, X2.shape[1], _ptr(X2), _ld(X2), _ptr(Y), _ld(Y)),
               "tlr_matvec")
        return Y if X.dim() == 2 else Y[:, 0]

    def info(self) -> dict:
        i = Info()
        _check(_load().tlr_get_info(self.h, C.byref(i)), "tlr_get_info")
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def ranks(self) -> np.ndarray:
        nb = self.info()["nb"]
        r = np.zeros((nb, nb), dtype=np.int32)
        _check(_load().tlr_get_ranks(self.ctx.h, self.h, r.ctypes.data), "tlr_get_ranks")
        return r

    def perm(self) -> np.ndarray:
        p = np.zeros(self.info()["N"], dtype=np.int64)
        _check(_load().tlr_get_perm(self.h, p.ctypes.data), "tlr_get_perm")
        return p

    def tile(self, i: int, j: int):
        """Host copies: diagonal (L_kk or A_kk, and D_k for LDL^T) or (U_ij, V_ij)."""
        inf = self.info()
        b = inf["b"]
        if i == j:
            U = np.zeros((b, b), order="F")
            V = np.zeros(b)
            _check(_load().tlr_get_tile(self.ctx.h, self.h, i, j, U.ctypes.data, V.ctypes.data), "tlr_get_tile")
            return U, (V if inf["state"] == 2 else None)
        r = int(self.ranks()[i, j])
        U = np.zeros((b, r), order="F")
        V = np.zeros((b, r), order="F")
        _check(_load().tlr_get_tile(self.ctx.h, self.h, i, j, U.ctypes.data if r else 0,
                                    V.ctypes.data if r else 0) if r else OK, "tlr_get_tile")
        return U, V
