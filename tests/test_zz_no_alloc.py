"""fram_sdsn_static: the SDSN entry point for callers that cannot allocate
device memory (their memory belongs to another allocator, or they cannot
afford cudaFree's device-wide synchronisation).  It must give the same result
as fram_sdsn, which runs the same kernel with context-owned scratch, on two
calls in a row (the static scratch keeps the previous call's contents), and
must reject sizes beyond its static limit with a message.

This file is collected last so that a failure here, under ``-x``, comes after
every other test has run.
"""
import numpy as np
import pytest

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


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,theta,cap", [(300, 10.0, 200), (1000, 2.0, 50), (97, 2.0, 5000)])
def test_static_matches_context_entry_twice(torch_cuda, ctx, n, theta, cap):
    torch = torch_cuda
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                      # two calls in a row share the scratch
        X = np.random.default_rng(100 * n + call).random((n, n)) ** 2
        Xd = torch.from_numpy(X).cuda()
        D_ref = torch.empty_like(Xd)
        D_sta = torch.empty_like(Xd)
        _, sw_ref, g_ref = fr.fram_sdsn(ctx, n, Xd, D_ref, theta, 1e-14, cap)
        st, sw, g, msg = fr.fram_sdsn_static(n, Xd, D_sta, theta, 1e-14, cap, stream)
        assert st == fr.FRAM_OK and msg == ""
        assert sw == sw_ref
        assert relF(D_sta.cpu().numpy(), D_ref.cpu().numpy()) <= 1e-12
        assert abs(g - g_ref) <= 1e-12 * max(1.0, abs(g_ref))


def test_static_rejects_sizes_beyond_limit(torch_cuda):
    torch = torch_cuda
    n = fr.FRAM_SDSN_STATIC_MAX_N + 1
    X = torch.zeros(1, dtype=torch.float64, device="cuda")   # never read: rejected first
    st, _, _, msg = fr.fram_sdsn_static(n, X, X, 2.0, check=False)
    assert st == fr.FRAM_ERR_INVALID
    assert "static scratch limit" in msg and str(fr.FRAM_SDSN_STATIC_MAX_N) in msg
