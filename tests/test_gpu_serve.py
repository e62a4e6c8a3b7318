"""Serving (fram_submit / fram_poll, continuous batching) through the C ABI.

A request's result must not depend on the other requests it shares ticks
with: every request keeps the SDSN sub-grid it would get alone and the same
kernels, so served results are compared with solo fram_solve results bit for
bit."""
import time

import numpy as np
import pytest

import fram_inputs as fi
import oracle as o
import paper_2508_00887_gb300 as fr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2508_00887_gb300 import build
    build.build()
    fr.load()
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    c = fr.fram_create(0, 0, torch_cuda.cuda.current_stream().cuda_stream)
    yield c
    fr.fram_destroy(c)


def solo(torch, ctx, g, params):
    X = torch.empty((g.n, g.n), dtype=torch.float64, device="cuda")
    P = torch.empty(g.n, dtype=torch.int32, device="cuda")
    _, info = fr.fram_solve(ctx, g.n, torch.from_numpy(g.A).cuda(), torch.from_numpy(g.B).cuda(),
                            None, params, X, P)
    return X.cpu().numpy(), P.cpu().numpy(), info


def test_served_equals_solo_in_a_mix(torch_cuda, ctx):
    torch = torch_cuda
    F, BF, TF = fr.FRAM_PREC_FP64, fr.FRAM_PREC_MIXED_BF16, fr.FRAM_PREC_MIXED_TF32
    specs = [(30, F), (80, F), (150, F), (300, F), (40, BF), (100, BF), (257, BF), (600, BF),
             (64, TF), (500, TF), (1000, BF)]
    reqs = []
    for k, (n, prec) in enumerate(specs):
        g = fi.er_pair(n, min(1.0, 12.0 / n), noise=0.05, seed=100 + k, theta=10.0)
        p = fr.fram_default_params(theta=10.0, precision=prec, max_polish=4 if prec != F else 0)
        # device inputs for some, host for others
        A = torch.from_numpy(g.A).cuda() if k % 2 else g.A
        B = torch.from_numpy(g.B).cuda() if k % 2 else g.B
        _, t = fr.fram_submit(ctx, n, A, B, p)
        reqs.append((g, p, t))
    for g, p, t in reqs:
        X = np.empty((g.n, g.n))
        P = np.empty(g.n, dtype=np.int32)
        st, info = fr.fram_poll(ctx, t, X, P, wait_ms=-1)
        assert st == fr.FRAM_OK
        Xs, Ps, si = solo(torch, ctx, g, p)
        assert info.outer_iters == si.outer_iters, g.meta
        assert np.array_equal(X, Xs), g.meta
        assert np.array_equal(P, Ps)
        assert info.objective == si.objective
        assert info.total_sweeps == si.total_sweeps
        assert info.ms_total > 0


def test_poll_semantics(torch_cuda, ctx):
    g = fi.medium_er_pair(3)
    p = fr.fram_default_params(theta=10.0, precision=fr.FRAM_PREC_MIXED_BF16, max_polish=4)
    _, t = fr.fram_submit(ctx, g.n, g.A, g.B, p)
    st, _ = fr.fram_poll(ctx, t, wait_ms=0, check=False)
    assert st in (fr.FRAM_NOT_READY, fr.FRAM_OK)
    if st == fr.FRAM_NOT_READY:
        st, _ = fr.fram_poll(ctx, t, None, np.empty(g.n, np.int32), wait_ms=-1)
        assert st == fr.FRAM_OK
    st, _ = fr.fram_poll(ctx, t, wait_ms=0, check=False)       # already retired
    assert st == fr.FRAM_ERR_INVALID
    st, _ = fr.fram_poll(ctx, 987654321, wait_ms=0, check=False)
    assert st == fr.FRAM_ERR_INVALID


def test_served_invalid_and_degenerate_requests(torch_cuda, ctx):
    g = fi.small_er_pair(4)
    bad = g.A.copy()
    bad[0, 1] += 1.0
    _, t1 = fr.fram_submit(ctx, g.n, bad, g.B)
    z = np.zeros((g.n, g.n))
    _, t2 = fr.fram_submit(ctx, g.n, z, z)
    _, t3 = fr.fram_submit(ctx, g.n, g.A, g.B)
    st1, _ = fr.fram_poll(ctx, t1, wait_ms=-1, check=False)
    st2, _ = fr.fram_poll(ctx, t2, wait_ms=-1, check=False)
    st3, info = fr.fram_poll(ctx, t3, None, np.empty(g.n, np.int32), wait_ms=-1)
    assert st1 == fr.FRAM_ERR_INVALID and st2 == fr.FRAM_ERR_DEGENERATE and st3 == fr.FRAM_OK


def test_admission_refused_when_budget_is_too_small(torch_cuda):
    torch = torch_cuda
    c = fr.fram_create(0, 64 * 1024, torch.cuda.current_stream().cuda_stream)
    try:
        g = fi.er_pair(200, 0.1, seed=1)
        _, t = fr.fram_submit(c, g.n, g.A, g.B)
        st, _ = fr.fram_poll(c, t, wait_ms=-1, check=False)
        assert st == fr.FRAM_ERR_OOM
        assert "budget" in fr.fram_last_error(c)
    finally:
        fr.fram_destroy(c)


def test_stream_of_requests_sampled_against_oracle(torch_cuda, ctx):
    # Poisson arrivals with log-uniform n in [20, 400]; all requests are in
    # flight together; a sample is re-solved by the oracle.
    times, specs = fi.serving_stream(60, seed=5, n_min=20, n_max=400, rate=2000.0)
    p = fr.fram_default_params(theta=10.0, precision=fr.FRAM_PREC_MIXED_BF16, max_polish=4)
    pairs, tickets = [], []
    t0 = time.perf_counter()
    for at, (n, seed) in zip(times, specs):
        while time.perf_counter() - t0 < at:
            pass
        g = fi.serving_pair(n, seed)
        _, t = fr.fram_submit(ctx, n, g.A, g.B, p)
        pairs.append(g)
        tickets.append(t)
    results = []
    for g, t in zip(pairs, tickets):
        P = np.empty(g.n, np.int32)
        st, info = fr.fram_poll(ctx, t, None, P, wait_ms=-1)
        assert st == fr.FRAM_OK
        assert sorted(P.tolist()) == list(range(g.n))
        results.append((P.astype(np.int64), info))
    for k in range(0, len(pairs), 15):
        g = pairs[k]
        ref = o.fram(g.A, g.B, theta=10.0)
        P, info = results[k]
        # equal accuracy, both ways
        assert abs(o.accuracy(P, g.truth) - o.accuracy(ref.perm, g.truth)) <= 0.005
        assert abs(info.objective - ref.objective) <= 1e-3 * abs(ref.objective)
