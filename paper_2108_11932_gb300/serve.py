"""Continuous-batching server for factor + solve + logdet requests.

Each request asks for the TLR Cholesky (or LDL^T) of a synthetic covariance
matrix (N points in [0,1]^d, exponential kernel with length scale ell), a solve
with nrhs right-hand sides and the log-determinant -- the unit of work of a
Gaussian-process likelihood sweep (Section 1 motivates the factorization by
such likelihoods).  Requests arrive over time and are submitted to the
library's serving queue, which admits them by its device bytes against the
context's HBM budget, builds their TLR matrices and adds them to one
factorization session: a request joins the in-flight batch at the next column
step, so its work overlaps on the device with the requests already running
(continuous batching).  Latency = arrival to result.

All GPU work and the admission, retry and request bookkeeping run in the
library; this module only generates the workload and submits at arrival times.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

import inputs


@dataclass
class Request:
    rid: int
    N: int
    d: int
    ell: float
    eps: float
    nrhs: int
    seed: int
    arrival: float
    b: int = 256
    admitted: float = -1.0
    finished: float = -1.0
    logdet: float = float("nan")
    status: int = 0
    est_bytes: int = 0
    result: np.ndarray | None = field(default=None, repr=False)


def tile_size(N: int) -> int:
    """Tile size growing as O(N^0.5) (Section 6, tile-size discussion): ~2 sqrt(N), power of two, 128..1024."""
    return int(min(1024, max(128, 2 ** round(math.log2(2.0 * math.sqrt(N))))))


def make_requests(n: int, rate: float, seed: int, n_min: int = 4096, n_max: int = 65536,
                  eps_choices=(1e-2, 1e-4, 1e-6), nrhs_max: int = 32) -> list[Request]:
    """Poisson arrivals at `rate`/s; N log-uniform in [n_min, n_max] rounded to a multiple of 256;
    d in {2, 3}; ell ~ U[0.05, 0.3]; eps from eps_choices; nrhs ~ U{1..nrhs_max}."""
    u = inputs.uniform(seed, 7, 6 * n).reshape(n, 6)
    t = 0.0
    out = []
    for r in range(n):
        t += -math.log(1.0 - u[r, 0]) / rate
        N = int(round(math.exp(math.log(n_min) + u[r, 1] * (math.log(n_max) - math.log(n_min))) / 256.0)) * 256
        N = min(max(N, n_min), n_max)
        d = 2 if u[r, 2] < 0.5 else 3
        ell = 0.05 + 0.25 * u[r, 3]
        eps = eps_choices[min(int(u[r, 4] * len(eps_choices)), len(eps_choices) - 1)]
        nrhs = 1 + min(int(u[r, 5] * nrhs_max), nrhs_max - 1)
        out.append(Request(r, N, d, ell, eps, nrhs, 1000 + r, t, b=tile_size(N)))
    return out


class Server:
    """Drives the library's serving queue (tlr_submit / tlr_progress / tlr_poll) with requests that
    arrive over time.  The library admits them by its device bytes against the context's HBM budget,
    factors them in one continuous batch, retries a loss of definiteness with a diagonal shift, and
    solves and takes the logdet; this loop only submits at arrival times and collects results."""

    def __init__(self, ctx, precision: int = 0, bs: int = 16, nugget: float = 1e-4):
        self.ctx = ctx
        self.precision = precision
        self.bs = bs
        self.nugget = nugget

    def run(self, requests: list[Request], keep_results: bool = False) -> dict:
        import paper_2108_11932_gb300 as T
        ctx = self.ctx
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        active: dict[int, Request] = {}
        steps = 0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                o = T.default_opts(bs=self.bs, seed=r.seed, precision=self.precision)
                x = inputs.points(r.N, r.d, r.seed)
                active[ctx.submit(x, r.b, r.eps, r.ell, self.nugget, inputs.rhs(r.N, r.nrhs, r.seed), o)] = r
            if not active:
                time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
                continue
            ctx.progress()
            steps += 1
            for t in list(active):
                got = ctx.poll(t, active[t].N, active[t].nrhs)
                if got is None:
                    continue
                r = active.pop(t)
                res, X = got
                r.finished = time.perf_counter() - t0
                r.admitted = r.finished - res["run_s"]
                r.status, r.logdet, r.retried = res["status"], res["logdet"], bool(res["retried"])
                r.est_bytes = res["bytes"]
                if keep_results:
                    r.result = X
        wall = time.perf_counter() - t0
        lat = np.array([r.finished - r.arrival for r in requests])
        wait = np.array([max(r.admitted - r.arrival, 0.0) for r in requests])
        ok = sum(1 for r in requests if r.status == 0)
        retried = sum(1 for r in requests if getattr(r, "retried", False))
        return {"requests": len(requests), "ok": ok, "shift_retries": retried, "wall_s": wall,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "throughput_req_s": len(requests) / wall,
                "queue_wait_p50_s": float(np.percentile(wait, 50)), "steps": steps}
