"""The library's serving queue (tlr_submit / tlr_progress / tlr_poll): continuous batching of
factor + solve + logdet requests admitted by an HBM budget.

A request's result must not depend on the requests it shares the device with: each matrix of the
shared batch keeps its own Gaussian stream, column index and split-K rule, so a request that joins
while others are in flight gets, bit for bit, the factor, solution and log determinant it gets
alone (compress -> potrf / ldlt -> solve -> logdet on its own).
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

MIX = [  # N, d, ell, b, eps, ldl, nrhs, seed
    (2048, 2, 0.1, 256, 1e-6, False, 3, 51),
    (1536, 3, 0.2, 256, 1e-4, True, 1, 52),
    (3072, 2, 0.05, 256, 1e-2, False, 5, 53),
    (1024, 3, 0.3, 128, 1e-6, False, 2, 54),
    (2560, 2, 0.15, 256, 1e-4, True, 4, 55),
    (1280, 2, 0.1, 128, 1e-2, False, 1, 56),
]


@pytest.fixture(scope="module")
def T():
    import paper_2108_11932_gb300 as T
    T.build()
    return T


def _alone(T, ctx, r):
    import torch
    N, d, ell, b, eps, ldl, nrhs, seed = r
    o = T.default_opts(bs=16, seed=seed)
    A = ctx.compress(inputs.points(N, d, seed), b, eps, ell, 1e-4, o)
    (A.ldlt if ldl else A.potrf)(eps, o)
    Bt = T.fortran(torch.tensor(inputs.rhs(N, nrhs, seed), device="cuda:0"))
    A.solve(Bt)
    ld, sg = A.logdet()
    out = (ld, sg, Bt.cpu().numpy(), A.info()["mean_rank"])
    A.free()
    return out


def _serve(T, ctx, mix, first_wave):
    """Submit the first `first_wave` requests, step twice, then submit the rest (they join the running
    batch); progress until done.  Returns results in request order and the largest in-flight count."""
    tickets, results, max_fl = {}, {}, 0

    def submit(i):
        N, d, ell, b, eps, ldl, nrhs, seed = mix[i]
        tickets[i] = ctx.submit(inputs.points(N, d, seed), b, eps, ell, 1e-4, inputs.rhs(N, nrhs, seed),
                                T.default_opts(bs=16, seed=seed), ldl=ldl)

    for i in range(first_wave):
        submit(i)
    for _ in range(2):
        q, fl = ctx.progress()
        max_fl = max(max_fl, fl)
    for i in range(first_wave, len(mix)):
        submit(i)
    while len(results) < len(mix):
        q, fl = ctx.progress()
        max_fl = max(max_fl, fl)
        for i, t in tickets.items():
            if i in results:
                continue
            got = ctx.poll(t, mix[i][0], mix[i][6])
            if got is not None:
                results[i] = got
        assert q >= 0 and fl >= 0
    return [results[i] for i in range(len(mix))], max_fl


def test_requests_in_the_mix_equal_their_alone_results(T):
    ctx = T.Context(0)
    alone = [_alone(T, ctx, r) for r in MIX]
    served, max_fl = _serve(T, ctx, MIX, first_wave=3)
    assert max_fl >= 3  # requests overlapped on the device
    for (res, X), (ld, sg, Xa, mr), r in zip(served, alone, MIX):
        assert res["status"] == 0 and not res["retried"], (r, res)
        assert res["logdet"] == ld and res["sign"] == sg, (r, res["logdet"], ld)
        assert np.array_equal(X, Xa), r
        assert res["mean_rank"] == mr and res["bytes"] > 0
    ctx.close()


def test_hbm_budget_admits_one_request_at_a_time_when_tight(T):
    """A budget below one request's footprint: the queue still admits a request whenever nothing is in
    flight, never more, and the results stay those of the requests alone."""
    ctx = T.Context(0, hbm_budget=1)
    mix = MIX[:4]
    alone = [_alone(T, ctx, r) for r in mix]
    served, max_fl = _serve(T, ctx, mix, first_wave=2)
    assert max_fl == 1
    for (res, X), (ld, sg, Xa, _), r in zip(served, alone, mix):
        assert res["status"] == 0 and res["logdet"] == ld and np.array_equal(X, Xa), r
    ctx.close()


def test_poll_releases_a_finished_request_and_rejects_unknown_tickets(T):
    ctx = T.Context(0)
    N, d, ell, b, eps, ldl, nrhs, seed = MIX[5]
    t = ctx.submit(inputs.points(N, d, seed), b, eps, ell, 1e-4, inputs.rhs(N, nrhs, seed),
                   T.default_opts(bs=16, seed=seed))
    got = None
    while got is None:
        ctx.progress()
        got = ctx.poll(t, N, nrhs)
    with pytest.raises(T.TLRError) as ei:
        ctx.poll(t, N, nrhs)
    assert ei.value.status == T.ERR_ARG
    # another ARA block width than the queue's first request is rejected
    with pytest.raises(T.TLRError) as ei:
        ctx.submit(inputs.points(N, d, seed), b, eps, ell, 1e-4, None, T.default_opts(bs=32, seed=seed))
    assert ei.value.status == T.ERR_ARG
    ctx.close()
