"""Acceptance values of the SVD oracle at full workload size (writes tests/golden/acceptance_<workload>.json).

Runs the oracle only (`oracle/`, with the seeded inputs of `inputs/`): for each threshold eps it
builds the TLR matrix with truncated-SVD tiles, factors it as L L^T and as L D L^T with every
column update formed densely and re-truncated by SVD (Algorithms 6 and 10), and records what
Section 6 checks for every result:

  * backward error ||A - L L^T||_2 / ||A||_2 (or L D L^T) by 30 power iterations from the Gaussian
    start vector of seed 12345, with the exact kernel matrix A applied on the fly;
  * relative residual ||A x - y||_2 / ||y||_2 of the solve with one N(0,1) right-hand side
    (stream 1 of the workload's seed);
  * log det of the factor.

A factorization that breaks down (a tile that is not positive definite) is retried once with the
diagonal shift eps I of Section 5.1, and the record says so.

Usage (about 2 hours for cov2d_131k on 8 cores, 10 minutes for cov3d_32k):
  python tests/golden/make_acceptance.py --workload cov2d_131k --eps 1e-2 1e-6
  python tests/golden/make_acceptance.py --workload cov3d_32k --eps 1e-4 1e-8
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import platform
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
from oracle import cmatvec, dense, measures, tlr  # noqa: E402

POWER_ITERS = 30
POWER_SEED = 12345


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _rank_stats(F) -> dict:
    r = np.array([u.shape[1] for u in F.U.values()], dtype=np.int64)
    return dict(mean=float(r.mean()) if r.size else 0.0, max=int(r.max()) if r.size else 0,
                total=int(r.sum()))


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", required=True, choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--eps", type=float, nargs="+", required=True)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1,
                    help="threads visiting the independent tiles of a column (BLAS runs one thread each)")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from threadpoolctl import threadpool_limits

    w = inputs.WORKLOADS[args.workload]
    N, d, ell, nug, b, seed = w["N"], w["d"], w["ell"], w["nugget"], w["b"], w["seed"]
    pts = inputs.points(N, d, seed)
    y = inputs.rhs(N, 1, seed)[:, 0]
    x0 = inputs.start_vector(N, POWER_SEED)
    t_all = time.perf_counter()
    out = dict(workload=args.workload, N=N, d=d, ell=ell, nugget=nug, b=b, seed=seed, compressor="svd",
               power=dict(iters=POWER_ITERS, seed=POWER_SEED, start="inputs.start_vector(N, 12345)"),
               rhs="inputs.rhs(N, 1, seed)", results={})
    factors = {}
    with ThreadPoolExecutor(args.threads) as pool, threadpool_limits(1):
        for eps in args.eps:
            key = f"{eps:g}"
            res = out["results"].setdefault(key, {})
            t0 = time.perf_counter()
            A = tlr.build(pts, b, eps, ell, nug, compressor="svd", mapper=pool.map)
            t_build = time.perf_counter() - t0
            res["build"] = dict(seconds=t_build, ranks=_rank_stats(A))
            print(f"[{args.workload} eps={key}] build {t_build:.0f} s, mean rank {res['build']['ranks']['mean']:.2f}",
                  flush=True)
            for kind in ("chol", "ldlt"):
                t0 = time.perf_counter()
                comp = None
                try:
                    F = tlr.factor(A, eps, ldl=(kind == "ldlt"), compressor="svd", mapper=pool.map)
                except dense.NotPositiveDefinite as ex:
                    comp = dict(kind="shift", shift=eps, first_failure_tile=int(getattr(ex, "tile", -1)))
                    F = tlr.factor(A, eps, ldl=(kind == "ldlt"), compressor="svd", compensation="shift",
                                   shift=eps, mapper=pool.map)
                t_fac = time.perf_counter() - t0
                t0 = time.perf_counter()
                xs = tlr.solve(F, y)
                t_solve = time.perf_counter() - t0
                rec = dict(compensation=comp, factor_seconds=t_fac, solve_seconds=t_solve, ranks=_rank_stats(F),
                           logdet=tlr.logdet(F))
                res[kind] = rec
                factors[(key, kind)] = (F, xs)
                print(f"[{args.workload} eps={key}] {kind}: factor {t_fac:.0f} s, mean rank "
                      f"{rec['ranks']['mean']:.2f}, logdet {rec['logdet']:.10g}", flush=True)
            del A

    # One pass of the exact kernel matrix per iteration serves every power iteration at once:
    # column 0 estimates ||A||_2, the others ||A - F||_2 of each factor F.
    keys = list(factors)
    t0 = time.perf_counter()
    AX = cmatvec.matvec(pts, ell, nug, np.stack([y] + [factors[k][1][:, 0] for k in keys], axis=1))
    for c, k in enumerate(keys, start=1):
        out["results"][k[0]][k[1]]["residual"] = float(np.linalg.norm(AX[:, c] - y) / np.linalg.norm(y))
    t_res = time.perf_counter() - t0

    def apply_block(V):
        W = cmatvec.matvec(pts, ell, nug, V)
        for c, k in enumerate(keys, start=1):
            W[:, c] -= tlr.matvec(factors[k][0], V[:, c:c + 1], "LLt")[:, 0]
        return W

    t0 = time.perf_counter()
    lam = measures.power_norms(apply_block, np.repeat(x0[:, None], 1 + len(keys), axis=1), POWER_ITERS)
    t_pow = time.perf_counter() - t0
    out["normA"] = float(lam[0])
    for c, k in enumerate(keys, start=1):
        r = out["results"][k[0]][k[1]]
        r["normE"] = float(lam[c])
        r["backward_error"] = float(lam[c] / lam[0])
        print(f"[{args.workload} eps={k[0]}] {k[1]}: backward error {r['backward_error']:.3e}, "
              f"residual {r['residual']:.3e}", flush=True)
    out["provenance"] = dict(
        script="tests/golden/make_acceptance.py",
        command="python tests/golden/make_acceptance.py --workload %s --eps %s" % (
            args.workload, " ".join(f"{e:g}" for e in args.eps)),
        date=datetime.datetime.now(datetime.timezone.utc).isoformat(timespec="seconds"),
        host=dict(cpu=_cpu_model(), machine=platform.machine(), cores=os.cpu_count(), tile_threads=args.threads,
                  matvec_threads=cmatvec.threads()),
        numpy=np.__version__, seconds_total=time.perf_counter() - t_all, seconds_residual=t_res,
        seconds_power=t_pow)
    path = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"acceptance_{args.workload}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote", path, flush=True)


if __name__ == "__main__":
    main()
