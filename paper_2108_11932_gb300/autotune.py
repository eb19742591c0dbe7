"""Autotuner for TLR factorizations on this GPU: tile size b, ARA block width bs, batch width.

Section 6 (Table 1) shows the best tile size depends on the problem (rank
distribution and size), and Section 7 names autotuning the tile size as future
work; the ARA block width (Algorithm 1's bs) and the dynamic-batch width
(Algorithm 5's subset size, `max_slots`) trade per-round work against the
number of rounds and launches.  The tuner times the factorization of one
representative synthetic covariance matrix per problem class (dimension d, size
bucket N) on the GPU at hand, by coordinate search: b at bs = 16 and full
width, then bs at the best b, then the width at the best (b, bs).  All work runs
through the library (construction and factorization kernels); the tuner only
picks among measured candidates.  None of the choices changes a factor's
accuracy contract (every rank is set by the threshold), and the batch width does
not change any result (the batched ARA is bitwise independent of it).
"""
from __future__ import annotations

import math
import time

import inputs

DEFAULT = (256, 16, 0)  # (b, bs, max_slots); max_slots 0: every tile of the column at once


def size_bucket(N: int) -> int:
    return int(round(math.log2(max(N, 1))))


def _time_factor(ctx, x, b, bs, width, eps, ell, nugget, seed, repeats):
    import torch

    import paper_2108_11932_gb300 as T
    o = T.default_opts(bs=bs, seed=seed, max_slots=width)
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
    return min(ts)


def tune(ctx, dims=(2, 3), sizes=(2048, 4096, 8192, 16384), candidates=(128, 256), bs_candidates=(16, 32),
         width_candidates=(0, 16), eps=1e-6, ell=0.15, nugget=1e-4, seed=97, repeats=2) -> dict:
    """Return {"table": {(d, size_bucket): (b, bs, max_slots)}, "timings": {(d, N, b, bs, width): s}}."""
    table, timings = {}, {}
    for d in dims:
        for N in sizes:
            x = inputs.points(N, d, seed)

            def measure(b, bs, width):
                key = (d, N, b, bs, width)
                if key not in timings:
                    timings[key] = _time_factor(ctx, x, b, bs, width, eps, ell, nugget, seed, repeats)
                return timings[key]

            bs0, w0 = bs_candidates[0], width_candidates[0]
            bb = [b for b in candidates if b <= N and bs0 <= b] or [min(N, DEFAULT[0])]
            b = min(bb, key=lambda v: measure(v, bs0, w0))
            bs = min([v for v in bs_candidates if v <= b], key=lambda v: measure(b, v, w0))
            width = min(width_candidates, key=lambda v: measure(b, bs, v))
            table[(d, size_bucket(N))] = (b, bs, width)
    return {"table": table, "timings": timings}


def choose(table: dict, N: int, d: int, default: tuple = DEFAULT) -> tuple:
    """(b, bs, max_slots) for a problem: the tuned class with the same d and the nearest size bucket."""
    cands = [(abs(k[1] - size_bucket(N)), k[1], v) for k, v in table.items() if k[0] == d]
    return tuple(min(cands)[2]) if cands else default
