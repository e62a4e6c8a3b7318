"""Full-size parity: n = 8192, the dense Gaussian workload's size, through
the same entry points and launch configurations the bench times.  The oracle
cannot afford every output at this size, so it computes sampled outputs one
by one (gradient columns), whole outputs where its cost is O(n^2) per step
(a few SDSN sweeps, the objective), and the rest is checked through
properties that hold at any size or through optima fixed by construction."""
import numpy as np
import pytest

import fram_inputs as fi
import oracle as o
import paper_2508_00887_gb300 as fr

pytestmark = pytest.mark.gpu

N_FULL = 8192


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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sym_random(rng, n):
    M = rng.random((n, n))
    M += M.T
    return M


def test_gradient_fp64_full_size_sampled_columns(torch_cuda, ctx):
    # Dense A and B (no sparse switch): the FP64 GEMM path of eq. 3 at n = 8192,
    # 16 sampled columns (a ragged spread across tiles) against the oracle.
    torch = torch_cuda
    n = N_FULL
    rng = np.random.default_rng(8192)
    A, B = sym_random(rng, n), sym_random(rng, n)
    N = rng.random((n, n)) / n
    K = rng.random((n, n))
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    fr.fram_gradient(ctx, n, dev(torch, A), dev(torch, N), dev(torch, B), X, dev(torch, K), 0.7)
    cols = np.unique(np.concatenate([[0, 127, 128, n - 1], rng.integers(0, n, 12)]))
    Xg = X[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    ref = o.gradient_columns(A, N, B, cols, K, 0.7)
    assert relF(Xg, ref) < 1e-13


def test_gradient_bf16_full_size_sampled_columns(torch_cuda, ctx):
    # The tcgen05 BF16 path at n = 8192 (the persistent 128 x 256 tiling): the
    # sampled columns sit within BF16 input rounding of the exact product.
    torch = torch_cuda
    n = N_FULL
    rng = np.random.default_rng(8193)
    A, B = sym_random(rng, n), sym_random(rng, n)
    N = rng.random((n, n)) / n
    X = torch.empty((n, n), dtype=torch.float32, device="cuda")
    fr.fram_gradient_lowp(ctx, n, dev(torch, A), dev(torch, N), dev(torch, B), X,
                          fr.FRAM_PREC_MIXED_BF16)
    cols = np.unique(np.concatenate([[0, 255, 256, n - 1], rng.integers(0, n, 12)]))
    Xg = X[:, torch.from_numpy(cols).cuda()].cpu().numpy().astype(np.float64)
    ref = o.gradient_columns(A, N, B, cols)
    assert relF(Xg, ref) < 1e-2
    assert np.all(np.isfinite(Xg))


def test_sdsn_fp64_full_size_three_sweeps_match_oracle(torch_cuda, ctx):
    # Three whole sweeps (each O(n^2) on the CPU) compared element by element.
    torch = torch_cuda
    n = N_FULL
    X = np.random.default_rng(8194).random((n, n)) ** 3
    ref = o.sdsn(X, 2.0, 1e-14, 3)
    Xd = dev(torch, X)
    Dd = torch.empty_like(Xd)
    _, sweeps, g = fr.fram_sdsn(ctx, n, Xd, Dd, 2.0, 1e-14, 3)
    D = Dd.cpu().numpy()
    assert sweeps == ref.sweeps == 3
    assert relF(D, ref.D) < 1e-12
    assert abs(g - ref.gamma) < 1e-12 * max(1.0, abs(ref.gamma))
    assert np.all(D >= 0)


def test_sdsn_fp64_full_size_capped_run_properties(torch_cuda, ctx):
    # The 200-sweep capped run: the reported gamma is sum(D)/n - 1 of the
    # returned matrix, D >= 0, and every row and column sum is within n gamma
    # of 1 from above (after the clamp each sum is >= 1 up to rounding).
    torch = torch_cuda
    n = N_FULL
    X = np.random.default_rng(8195).random((n, n)) ** 3
    Xd = dev(torch, X)
    _, sweeps, g = fr.fram_sdsn(ctx, n, Xd, Xd, 2.0, 1e-14, 200)
    D = Xd.cpu().numpy()
    assert 1 <= sweeps <= 200
    assert np.all(D >= 0)
    total = D.sum(dtype=np.float64)
    assert abs((total / n - 1.0) - g) <= 1e-12 + 1e-12 * abs(g)
    r, c = D.sum(1), D.sum(0)
    assert r.min() >= 1 - 1e-9 and c.min() >= 1 - 1e-9
    assert r.max() <= 1 + n * g + 1e-9 and c.max() <= 1 + n * g + 1e-9


def test_assign_full_size_planted_optimum(torch_cuda, ctx):
    # W_ij = a_i + b_j + eps [j = sigma(i)]: every permutation has the value
    # sum(a) + sum(b) plus eps per position it shares with sigma, so sigma is
    # the unique optimum.  b has a clear maximum, so nearly every row argmax
    # lands on one column and the cluster completion places 8191 rows.
    torch = torch_cuda
    n = N_FULL
    rng = np.random.default_rng(8196)
    a = rng.random(n)
    b = rng.random(n) * 0.5
    b[1234] = 2.0
    sigma = rng.permutation(n)
    eps = 1e-3
    W = a[:, None] + b[None, :]
    W[np.arange(n), sigma] += eps
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val = fr.fram_assign(ctx, n, dev(torch, W), perm)
    p = perm.cpu().numpy().astype(np.int64)
    assert np.array_equal(p, sigma)
    assert abs(val - W[np.arange(n), sigma].sum()) <= 1e-12 * n


def test_assign_random_4096_matches_oracle(torch_cuda, ctx):
    # Random W at the social workload's size class: about a third of the rows
    # lose their argmax column, and the shortest augmenting paths are long.
    torch = torch_cuda
    n = 4096
    W = np.random.default_rng(4096).random((n, n))
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val = fr.fram_assign(ctx, n, dev(torch, W), perm)
    p = perm.cpu().numpy().astype(np.int64)
    ref = o.lap_max(W)
    assert np.array_equal(p, ref)                 # unique optimum for random W
    assert abs(val - W[np.arange(n), ref].sum()) <= 1e-12 * n


def test_mixed_solve_full_size_properties(torch_cuda, ctx):
    # The bench's n = 8192 dense solve (BF16 GEMMs, FP32 SDSN, FP64 polish).
    # Checked at any size: the permutation is one; the reported objective is
    # the oracle's eq. 1 at that permutation on the unscaled inputs; N >= 0
    # and finite; the assignment value is sum_i N[i, perm(i)] and no larger
    # than the sum of row maxima; a second solve is bit-identical.
    torch = torch_cuda
    g = fi.large_gaussian_pair(0, n=N_FULL)
    n = g.n
    A, B = dev(torch, g.A), dev(torch, g.B)
    p = fr.fram_default_params(theta=g.theta, precision=fr.FRAM_PREC_MIXED_BF16, max_polish=4)

    def run():
        X = torch.empty((n, n), dtype=torch.float64, device="cuda")
        P = torch.empty(n, dtype=torch.int32, device="cuda")
        _, info = fr.fram_solve(ctx, n, A, B, None, p, X, P)
        return X, P.cpu().numpy().astype(np.int64), info

    X, P, info = run()
    assert sorted(P.tolist()) == list(range(n))
    assert abs(info.objective - o.objective(g.A, g.B, P)) <= 1e-9 * abs(info.objective)
    Nh = X.cpu().numpy()
    assert np.all(np.isfinite(Nh)) and np.all(Nh >= 0)
    chosen = Nh[np.arange(n), P].sum()
    assert abs(info.assignment_value - chosen) <= 1e-9 * abs(chosen)
    assert chosen <= Nh.max(axis=1).sum() + 1e-12 * n
    X2, P2, info2 = run()
    assert np.array_equal(P, P2) and bool(torch.equal(X, X2))
    assert info2.objective == info.objective and info2.outer_iters == info.outer_iters
