"""Sparse-graph gradient of the FP64 path (eq. 3 with CSR products): the
CSR products add the same terms in the same order as the dense GEMM, so
gradients and whole solves must be bit-identical with and without them,
and the sparse path must match the oracle like the dense one."""
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
    fr.fram_set_sparse_density(c, 0.2)
    fr.fram_destroy(c)


def gradient(torch, ctx, A, N, B, K=None, lam=0.7):
    n = A.shape[0]
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    d = lambda M: torch.from_numpy(M).cuda()
    fr.fram_gradient(ctx, n, d(A), d(N), d(B), X, d(K) if K is not None else None, lam)
    return X.cpu().numpy()


@pytest.mark.parametrize("n,p", [(64, 0.05), (200, 0.02), (333, 0.1)])
def test_sparse_gradient_bit_identical_to_dense(torch_cuda, ctx, n, p):
    g = fi.er_pair(n, p, noise=0.05, seed=n)
    N = np.random.default_rng(1).random((n, n))
    K = np.random.default_rng(2).random((n, n))
    fr.fram_set_sparse_density(ctx, 0.0)
    dense = gradient(torch_cuda, ctx, g.A, N, g.B, K)
    fr.fram_set_sparse_density(ctx, 1.0)
    sparse = gradient(torch_cuda, ctx, g.A, N, g.B, K)
    fr.fram_set_sparse_density(ctx, 0.2)
    assert np.array_equal(dense, sparse)
    ref = o.gradient(g.A, N, g.B, K, 0.7)
    assert np.linalg.norm(sparse - ref) <= 1e-14 * np.linalg.norm(ref)


def test_sparse_gradient_with_nearly_symmetric_b(torch_cuda, ctx):
    # B symmetric only to 1e-13: the CSR of B^T keeps the products equal to
    # T B exactly (not T B^T).
    g = fi.er_pair(150, 0.05, noise=0.05, seed=3)
    B = g.B.copy()
    nz = np.argwhere(np.triu(B, 1) > 0)[:20]
    for i, j in nz:
        B[i, j] *= 1 + 1e-13
    N = np.random.default_rng(4).random((150, 150))
    fr.fram_set_sparse_density(ctx, 0.0)
    dense = gradient(torch_cuda, ctx, g.A, N, B)
    fr.fram_set_sparse_density(ctx, 1.0)
    sparse = gradient(torch_cuda, ctx, g.A, N, B)
    fr.fram_set_sparse_density(ctx, 0.2)
    assert np.array_equal(dense, sparse)


def solve64(torch, ctx, g):
    n = g.n
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    _, info = fr.fram_solve(ctx, n, torch.from_numpy(g.A).cuda(), torch.from_numpy(g.B).cuda(),
                            None, fr.fram_default_params(theta=g.theta), X, P)
    return X.cpu().numpy(), P.cpu().numpy().astype(np.int64), info


def test_social_pair_solve_sparse_equals_dense_and_oracle(torch_cuda, ctx):
    g = fi.social_pair(400, 2200, 0.05, seed=2)
    fr.fram_set_sparse_density(ctx, 0.0)
    Xd, Pd, infod = solve64(torch_cuda, ctx, g)
    fr.fram_set_sparse_density(ctx, 0.2)
    Xs, Ps, infos = solve64(torch_cuda, ctx, g)
    assert np.array_equal(Xd, Xs) and np.array_equal(Pd, Ps)
    assert infod.outer_iters == infos.outer_iters
    ref = o.fram(g.A, g.B, theta=g.theta)
    assert infos.outer_iters == ref.outer_iters
    assert np.linalg.norm(Xs - ref.N) <= 1e-9 * np.linalg.norm(ref.N)
    assert np.array_equal(Ps, ref.perm)


def test_set_sparse_density_rejects_out_of_range(torch_cuda, ctx):
    assert fr.fram_set_sparse_density(ctx, -0.1, check=False) == fr.FRAM_ERR_INVALID
    assert fr.fram_set_sparse_density(ctx, 1.5, check=False) == fr.FRAM_ERR_INVALID
