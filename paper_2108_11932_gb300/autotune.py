"""Tile-size autotuner for TLR factorizations on this GPU.

Section 6 (Table 1) shows the best tile size depends on the problem (rank
distribution and size), and Section 7 names autotuning the tile size as future
work.  The tuner times the factorization of one representative synthetic
covariance matrix per problem class (dimension d, size bucket N) for each
candidate tile size b, on the GPU at hand, and keeps the fastest.  All work
runs through the library (construction and factorization kernels); the tuner
only picks among measured candidates.
"""
from __future__ import annotations

import math
import time

import inputs


def size_bucket(N: int) -> int:
    return int(round(math.log2(max(N, 1))))


def tune(ctx, dims=(2, 3), sizes=(2048, 4096, 8192, 16384), candidates=(128, 256), eps=1e-6, ell=0.15,
         nugget=1e-4, bs=16, seed=97, repeats=2) -> dict:
    """Return {(d, size_bucket): b} with the fastest candidate tile size per class."""
    import torch

    import paper_2108_11932_gb300 as T
    table, timings = {}, {}
    for d in dims:
        for N in sizes:
            x = inputs.points(N, d, seed)
            best = None
            for b in candidates:
                if b > N:
                    continue
                o = T.default_opts(bs=bs, seed=seed)
                A = ctx.compress(x, b, eps, ell, nugget, o)
                ts = []
                for _ in range(repeats):
                    F = A.copy()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    F.potrf(eps, o)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                    F.free()
                A.free()
                t = min(ts)
                timings[(d, N, b)] = t
                if best is None or t < best[1]:
                    best = (b, t)
            table[(d, size_bucket(N))] = best[0]
    return {"table": table, "timings": timings}


def choose(table: dict, N: int, d: int, default: int = 256) -> int:
    """Tile size for a problem: the tuned class with the same d and the nearest size bucket."""
    cands = [(abs(k[1] - size_bucket(N)), v) for k, v in table.items() if k[0] == d]
    return min(cands)[1] if cands else default
