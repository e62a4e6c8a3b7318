"""Node-attribute term (eq. 1 <N, F F~^T>, eq. 3 lambda F F~^T) through the C
ABI: fram_node_affinity against the oracle, and solves that use it against
the oracle's FRAM with the same K."""
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


def affinity_gpu(torch, ctx, F, Ft):
    n, d = F.shape
    K = torch.empty((n, n), dtype=torch.float64, device="cuda")
    fr.fram_node_affinity(ctx, n, d, torch.from_numpy(F).cuda(), torch.from_numpy(Ft).cuda(), K)
    return K


@pytest.mark.parametrize("n,d", [(1, 1), (5, 3), (64, 16), (130, 37), (1000, 128)])
def test_node_affinity_matches_oracle(torch_cuda, ctx, n, d):
    # Sizes cover one tile, several tiles and ragged edges in n and in d.
    rng = np.random.default_rng(n + d)
    F, Ft = rng.random((n, d)), rng.random((n, d))
    K = affinity_gpu(torch_cuda, ctx, F, Ft).cpu().numpy()
    ref = o.node_affinity(F, Ft)
    assert np.max(np.abs(K - ref)) <= 4 * d * np.finfo(float).eps * np.max(np.abs(ref))


def test_node_affinity_exact_on_dyadic_inputs(torch_cuda, ctx):
    # Small dyadic entries: every product and partial sum is exact, so the
    # GPU must agree with the oracle bit for bit whatever the order.
    rng = np.random.default_rng(3)
    F = rng.integers(0, 16, (70, 20)) / 16.0
    Ft = rng.integers(0, 16, (70, 20)) / 16.0
    K = affinity_gpu(torch_cuda, ctx, F, Ft).cpu().numpy()
    assert np.array_equal(K, o.node_affinity(F, Ft))


def test_node_affinity_rejects_bad_arguments(torch_cuda, ctx):
    torch = torch_cuda
    F = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    K = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    assert fr.fram_node_affinity(ctx, 4, 0, F, F, K, check=False) == fr.FRAM_ERR_INVALID
    assert fr.fram_node_affinity(ctx, 0, 2, F, F, K, check=False) == fr.FRAM_ERR_INVALID
    host = np.zeros((4, 2))
    assert fr.fram_node_affinity(ctx, 4, 2, host, F, K, check=False) == fr.FRAM_ERR_INVALID


def solve(torch, ctx, g, params):
    n, d = g.F.shape
    K = affinity_gpu(torch, ctx, g.F, g.Ft)
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    _, info = fr.fram_solve(ctx, n, torch.from_numpy(g.A).cuda(), torch.from_numpy(g.B).cuda(),
                            K, params, X, P)
    return X.cpu().numpy(), P.cpu().numpy().astype(np.int64), info


def test_attributed_solve_matches_oracle(torch_cuda, ctx):
    # FP64 path with K from the GPU affinity; N(0) = 0 because K is given.
    g = fi.attributed_pair(200, d=32, seed=4)
    ref = o.fram(g.A, g.B, K=o.node_affinity(g.F, g.Ft), theta=2.0)
    X, P, info = solve(torch_cuda, ctx, g, fr.fram_default_params(theta=2.0))
    assert info.outer_iters == ref.outer_iters
    assert np.linalg.norm(X - ref.N) <= 1e-9 * np.linalg.norm(ref.N)
    assert np.array_equal(P, ref.perm)
    assert abs(info.objective - ref.objective) <= 1e-12 * abs(ref.objective)


def test_attributed_solve_mixed_equal_accuracy(torch_cuda, ctx):
    g = fi.attributed_pair(300, d=64, seed=5)
    ref = o.fram(g.A, g.B, K=o.node_affinity(g.F, g.Ft), theta=2.0)
    for prec in (fr.FRAM_PREC_MIXED_BF16, fr.FRAM_PREC_MIXED_TF32):
        p = fr.fram_default_params(theta=2.0, precision=prec, max_polish=4)
        _, P, info = solve(torch_cuda, ctx, g, p)
        assert o.accuracy(P, g.truth) >= o.accuracy(ref.perm, g.truth) - 0.005
        assert info.objective >= ref.objective - 1e-3 * abs(ref.objective)
