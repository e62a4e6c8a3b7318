"""Exact FRA projection (eq. 4 / Thm. 1; a variant of step 6) through the C
ABI.  The projection is unique (strictly convex QP), so the GPU result is
compared with the oracle's point by point within the stop tolerance, and on
its own with the KKT certificate (nonnegative, unit row and column sums)."""
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


def fram_iterate_X(n, theta, seed):
    g = fi.er_pair(n, min(1.0, 12.0 / n), noise=0.05, seed=seed, theta=theta)
    r = o.fram(g.A, g.B, theta=theta, max_outer=3)
    As, Bs, _, _ = o.prescale(g.A, g.B)
    return o.gradient(As, r.N, Bs)


@pytest.mark.parametrize("n,theta,seed", [(1, 10.0, 0), (7, 10.0, 1), (64, 10.0, 2),
                                          (200, 2.0, 3), (300, 10.0, 4), (1000, 10.0, 5)])
def test_fra_exact_matches_oracle(torch_cuda, ctx, n, theta, seed):
    torch = torch_cuda
    X = np.random.default_rng(seed).random((n, n)) if n < 60 else fram_iterate_X(n, theta, seed)
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    tol = 1e-11
    _, sweeps, res = fr.fram_fra_exact(ctx, n, torch.from_numpy(X).cuda(), D, theta, tol=tol)
    Dg = D.cpu().numpy()
    assert res <= tol and sweeps >= 1
    assert np.all(Dg >= 0)
    assert np.max(np.abs(Dg.sum(1) - 1)) <= 2 * tol
    assert np.max(np.abs(Dg.sum(0) - 1)) <= 1e-12 * max(1, n / 100)
    # Both points are within their residual of the unique projection.
    ref = o.fra_exact(X, theta, tol=1e-12 if n <= 300 else 1e-11, omega=1.6)
    assert ref.converged
    assert np.max(np.abs(Dg - ref.D)) <= 1e-8


@pytest.mark.parametrize("n", [1500, 2100])
def test_fra_exact_wide_rows(torch_cuda, ctx, n):
    # n = 1500 keeps each equation's keys in registers (64 per lane); n = 2100
    # is past that and streams Y0 on every Newton pass.  Random X: the
    # oracle finishes these sizes in seconds.
    torch = torch_cuda
    X = np.random.default_rng(n).random((n, n))
    D = torch.empty((n, n), dtype=torch.float64, device="cuda")
    tol = 1e-11
    _, sweeps, res = fr.fram_fra_exact(ctx, n, torch.from_numpy(X).cuda(), D, 10.0, tol=tol)
    Dg = D.cpu().numpy()
    assert res <= tol and sweeps >= 1
    assert np.all(Dg >= 0)
    assert np.max(np.abs(Dg.sum(1) - 1)) <= 2 * tol
    assert np.max(np.abs(Dg.sum(0) - 1)) <= 1e-12 * n / 100
    ref = o.fra_exact(X, 10.0, tol=tol, omega=1.6)
    assert ref.converged
    assert np.max(np.abs(Dg - ref.D)) <= 1e-8


def test_fra_exact_in_place_and_degenerate(torch_cuda, ctx):
    torch = torch_cuda
    n = 50
    X = np.random.default_rng(9).random((n, n))
    Xd = torch.from_numpy(X).cuda()
    fr.fram_fra_exact(ctx, n, Xd, Xd, 10.0)
    ref = o.fra_exact(X, 10.0, tol=1e-12)
    assert np.max(np.abs(Xd.cpu().numpy() - ref.D)) <= 1e-8
    Z = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st, _, _ = fr.fram_fra_exact(ctx, n, Z, Z, 10.0, check=False)
    assert st == fr.FRAM_ERR_DEGENERATE


def test_fra_exact_sweep_cap(torch_cuda, ctx):
    # With a cap of 3 sweeps the result is feasible in the columns but not
    # yet in the rows, and the call says so through the residual.
    torch = torch_cuda
    X = fram_iterate_X(300, 10.0, 4)
    D = torch.empty((300, 300), dtype=torch.float64, device="cuda")
    _, sweeps, res = fr.fram_fra_exact(ctx, 300, torch.from_numpy(X).cuda(), D, 10.0, tol=1e-12,
                                       max_sweeps=3)
    assert sweeps == 3 and res > 1e-12
    assert abs(np.max(np.abs(D.cpu().numpy().sum(1) - 1)) - res) <= 1e-9


def solve(torch, ctx, g, params):
    n = g.n
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    _, info = fr.fram_solve(ctx, n, torch.from_numpy(g.A).cuda(), torch.from_numpy(g.B).cuda(),
                            None, params, X, P)
    return X.cpu().numpy(), P.cpu().numpy().astype(np.int64), info


@pytest.mark.parametrize("seed", [0, 1])
def test_solve_with_exact_projection_matches_oracle(torch_cuda, ctx, seed):
    g = fi.small_er_pair(seed)
    p = fr.fram_default_params(theta=10.0, projection=fr.FRAM_PROJ_EXACT, max_sweeps=5000)
    X, P, info = solve(torch_cuda, ctx, g, p)
    ref = o.fram(g.A, g.B, theta=10.0, projection="exact", max_sweeps=5000, omega=1.6)
    assert info.outer_iters == ref.outer_iters
    assert np.linalg.norm(X - ref.N) <= 1e-8 * np.linalg.norm(ref.N)
    assert np.array_equal(P, ref.perm)
    assert info.gamma <= 8 * g.n * 2.0 ** -52
    assert o.accuracy(P, g.truth) == 1.0


def test_exact_projection_rejected_where_unsupported(torch_cuda, ctx):
    g = fi.small_er_pair(0)
    for prec in (fr.FRAM_PREC_MIXED_BF16, fr.FRAM_PREC_MIXED_TF32):
        p = fr.fram_default_params(projection=fr.FRAM_PROJ_EXACT, precision=prec)
        st, _ = fr.fram_solve(ctx, g.n, g.A, g.B, None, p, None, np.empty(g.n, np.int32),
                              check=False)
        assert st == fr.FRAM_ERR_INVALID
    p = fr.fram_default_params(projection=fr.FRAM_PROJ_EXACT)
    st, _ = fr.fram_solve_batched(ctx, [g.n], [g.A], [g.B], p, None,
                                  [np.empty(g.n, np.int32)], check=False)
    assert st == fr.FRAM_ERR_INVALID
    st, _ = fr.fram_submit(ctx, g.n, g.A, g.B, p, check=False)
    assert st == fr.FRAM_ERR_INVALID
