"""Continuous-batching server for factor + solve + logdet requests.

Each request asks for the TLR Cholesky (or LDL^T) of a synthetic covariance
matrix (N points in [0,1]^d, exponential kernel with length scale ell), a solve
with nrhs right-hand sides and the log-determinant -- the unit of work of a
Gaussian-process likelihood sweep (Section 1 motivates the factorization by
such likelihoods).  Requests arrive over time; the server admits an arrived
request when its estimated device footprint fits the memory budget, builds its
TLR matrix, and adds it to the factorization session: it joins the in-flight
batch at the next column step, so its work overlaps on the device with the
requests already running (continuous batching).  When its factorization
finishes the server solves and takes the logdet; the factor stays resident
until then and is released afterwards.  Latency = arrival to result.

All GPU work runs in the library; this module only schedules.
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


def footprint(req: Request, mean_rank: float = 48.0) -> int:
    """Device bytes of a request while in flight: dense diagonal tiles, their inverses and the
    working copy (3 N b), low-rank factors of A and L (2 x 2 (N^2/b)/2 r) and the ARA workspace."""
    nb = max(1, req.N // req.b)
    lowrank = 2 * 2 * (nb * (nb - 1) / 2) * req.b * mean_rank
    work = nb * req.b * (req.b + 32)
    return int(8 * (3 * req.N * req.b + lowrank + work + req.N * (req.nrhs + req.d)))


class Server:
    def __init__(self, ctx, budget_bytes: float = 150e9, precision: int = 0, bs: int = 16, nugget: float = 1e-4):
        self.ctx = ctx
        self.budget = budget_bytes
        self.precision = precision
        self.bs = bs
        self.nugget = nugget

    def run(self, requests: list[Request], keep_results: bool = False) -> dict:
        import torch

        import paper_2108_11932_gb300 as T
        ctx = self.ctx
        S = T.Session(ctx)
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        active: dict[int, tuple[Request, object]] = {}
        resident = 0
        steps = 0
        busy_s = 0.0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            # admission: arrived requests, in arrival order, while the budget allows
            while pending and pending[0].arrival <= now:
                r = pending[0]
                r.est_bytes = footprint(r)
                if active and resident + r.est_bytes > self.budget:
                    break
                pending.popleft()
                r.admitted = time.perf_counter() - t0
                x = inputs.points(r.N, r.d, r.seed)
                o = T.default_opts(bs=self.bs, seed=r.seed, precision=self.precision)
                A = ctx.compress(x, r.b, r.eps, r.ell, self.nugget, o)
                ticket = S.add(A, r.eps, o)
                active[ticket] = (r, A)
                resident += r.est_bytes
            if not active:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t0)))
                continue
            ts = time.perf_counter()
            S.step()
            steps += 1
            for t in list(active):
                fin, st = S.poll(t)
                if not fin:
                    continue
                r, A = active.pop(t)
                r.status = st
                if st != 0 and not getattr(r, "retried", False):
                    # loss of definiteness at a loose threshold: refactor A + eps I (Section 5.1,
                    # diagonal shift s <= eps), noted on the request
                    A.free()
                    r.retried = True
                    x = inputs.points(r.N, r.d, r.seed)
                    o = T.default_opts(bs=self.bs, seed=r.seed, precision=self.precision,
                                       compensation=T.COMP_SHIFT, shift=r.eps)
                    A = ctx.compress(x, r.b, r.eps, r.ell, self.nugget, o)
                    active[S.add(A, r.eps, o)] = (r, A)
                    continue
                if st == 0:
                    B = T.fortran(torch.tensor(inputs.rhs(r.N, r.nrhs, r.seed), device=f"cuda:{ctx.device}"))
                    A.solve(B)
                    r.logdet = A.logdet()[0]
                    if keep_results:
                        r.result = B.cpu().numpy()
                r.finished = time.perf_counter() - t0
                resident -= r.est_bytes
                A.free()
            busy_s += time.perf_counter() - ts
        wall = time.perf_counter() - t0
        S.close()
        lat = np.array([r.finished - r.arrival for r in requests])
        ok = sum(1 for r in requests if r.status == 0)
        retried = sum(1 for r in requests if getattr(r, "retried", False))
        return {"requests": len(requests), "ok": ok, "shift_retries": retried, "wall_s": wall,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "throughput_req_s": len(requests) / wall,
                "steps": steps, "step_busy_s": busy_s}
