"""GPU FP64 path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances: the oracle and the kernels sum in different orders, so values
agree to rounding (relative ~1e-15 per step) and the fixed-point iteration
does not amplify it (checked on the oracle: perturbing the inputs by 1e-15
moves the final N by ~2e-16).  The bar is the one the FP64 path targets:
relative Frobenius error of N <= 1e-9 and the identical permutation.
"""
import numpy as np
import pytest

import fram_inputs as fi
import oracle as o
import paper_2508_00887_gb300 as fr

pytestmark = pytest.mark.gpu

RTOL_N = 1e-9


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


def dev(torch, a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------ step level
@pytest.mark.parametrize("n", [5, 50, 97, 130, 300, 1000])
@pytest.mark.parametrize("theta", [2.0, 10.0])
def test_sdsn_matches_oracle(torch_cuda, ctx, n, theta):
    torch = torch_cuda
    rng = np.random.default_rng(n)
    X = rng.random((n, n)) ** 3
    ref = o.sdsn(X, theta, 1e-14, 200)
    Xd = dev(torch, X)
    Dd = torch.empty_like(Xd)
    _, sweeps, g = fr.fram_sdsn(ctx, n, Xd, Dd, theta, 1e-14, 200)
    D = Dd.cpu().numpy()
    if ref.converged:       # the stop test sits at the rounding floor of gamma
        assert abs(sweeps - ref.sweeps) <= 1
    else:                   # capped: the sweep count is part of the result
        assert sweeps == ref.sweeps
    assert relF(D, ref.D) < 1e-12
    assert abs(g - ref.gamma) < 1e-12 * max(1.0, abs(ref.gamma))
    assert np.all(D >= 0)


def test_sdsn_converged_is_doubly_stochastic(torch_cuda, ctx):
    torch = torch_cuda
    n = 150
    X = np.random.default_rng(1).random((n, n))
    ref = o.sdsn(X, 2.0, 1e-14, 5000)
    Xd = dev(torch, X)
    _, sweeps, g = fr.fram_sdsn(ctx, n, Xd, Xd, 2.0, 1e-14, 5000)   # in place
    D = Xd.cpu().numpy()
    assert ref.converged and g <= 1e-14
    assert abs(sweeps - ref.sweeps) <= 1            # stop test sits at the rounding floor
    assert np.max(np.abs(D.sum(0) - 1)) < 1e-12 and np.max(np.abs(D.sum(1) - 1)) < 1e-12
    assert relF(D, ref.D) < 1e-12


def test_sdsn_golden_2x2(torch_cuda, ctx):
    torch = torch_cuda
    X = dev(torch, np.eye(2))
    D = torch.empty_like(X)
    _, sweeps, g = fr.fram_sdsn(ctx, 2, X, D, 10.0, 1e-14, 200)
    assert sweeps == 49 and g == 2.0 ** -47
    assert np.array_equal(D.cpu().numpy(), np.diag([1 + 2.0 ** -47] * 2))


def test_sdsn_degenerate(torch_cuda, ctx):
    torch = torch_cuda
    X = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    st, _, _ = fr.fram_sdsn(ctx, 4, X, X, 2.0, check=False)
    assert st == fr.FRAM_ERR_DEGENERATE


@pytest.mark.parametrize("n", [1, 50, 129, 300])
def test_gradient_matches_oracle(torch_cuda, ctx, n):
    torch = torch_cuda
    rng = np.random.default_rng(7 + n)
    A = rng.random((n, n)); A = A + A.T
    B = rng.random((n, n)); B = B + B.T
    N = rng.random((n, n))
    K = rng.random((n, n))
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    fr.fram_gradient(ctx, n, dev(torch, A), dev(torch, N), dev(torch, B), X, dev(torch, K), 0.7)
    ref = o.gradient(A, N, B, K, 0.7)
    assert relF(X.cpu().numpy(), ref) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 7, 64, 300, 1000, 1100, 2100])
def test_assign_matches_oracle(torch_cuda, ctx, n):
    # n >= 1024 runs the cluster completion (1100 and 2100: ragged column
    # blocks); random W leaves about a third of the rows in conflict.
    torch = torch_cuda
    W = np.random.default_rng(n).random((n, n))
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val = fr.fram_assign(ctx, n, dev(torch, W), perm)
    p = perm.cpu().numpy().astype(np.int64)
    ref = o.lap_max(W)
    assert sorted(p.tolist()) == list(range(n))
    assert abs(val - W[np.arange(n), ref].sum()) <= 1e-12 * n
    assert np.array_equal(p, ref)                  # unique optimum for random W


def test_assign_conflicting_argmaxes(torch_cuda, ctx):
    # Every row prefers column 0 (and then a shared second choice), so the
    # argmax start leaves almost every row to the augmenting-path search.
    torch = torch_cuda
    n = 200
    rng = np.random.default_rng(3)
    W = rng.random((n, n)) * 0.5
    W[:, 0] += 1.0
    W[:, 1] += 0.8
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val = fr.fram_assign(ctx, n, dev(torch, W), perm)
    p = perm.cpu().numpy().astype(np.int64)
    ref = o.lap_max(W)
    assert sorted(p.tolist()) == list(range(n))
    assert abs(val - W[np.arange(n), ref].sum()) <= 1e-12 * n
    assert np.array_equal(p, ref)


def test_assign_ties_valid(torch_cuda, ctx):
    torch = torch_cuda
    n = 12
    W = np.kron(np.eye(4), np.ones((3, 3)))
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val = fr.fram_assign(ctx, n, dev(torch, W), perm)
    p = perm.cpu().numpy()
    assert sorted(p.tolist()) == list(range(n))
    assert abs(val - n) < 1e-12


@pytest.mark.parametrize("levels", [2, 4])
def test_assign_integer_ties_optimal_value(torch_cuda, ctx, levels):
    # Few distinct values: the row reduction meets tied minima at almost every
    # step.  The optimum value is unique even where the permutation is not.
    torch = torch_cuda
    n = 300
    W = np.random.default_rng(levels).integers(0, levels, (n, n)).astype(np.float64)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val = fr.fram_assign(ctx, n, dev(torch, W), perm)
    p = perm.cpu().numpy().astype(np.int64)
    ref = o.lap_max(W)
    assert sorted(p.tolist()) == list(range(n))
    assert W[np.arange(n), p].sum() == W[np.arange(n), ref].sum()
    assert val == W[np.arange(n), ref].sum()


def test_assign_constant_matrix(torch_cuda, ctx):
    torch = torch_cuda
    n = 500
    W = np.full((n, n), 0.25)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val = fr.fram_assign(ctx, n, dev(torch, W), perm)
    assert sorted(perm.cpu().numpy().tolist()) == list(range(n))
    assert val == 0.25 * n


def test_assign_diffuse_doubly_stochastic(torch_cuda, ctx):
    # A near-uniform doubly stochastic matrix, as FRAM produces at small theta
    # on large pairs: almost every argmax conflicts.
    torch = torch_cuda
    n = 1500
    rng = np.random.default_rng(11)
    W = 1.0 + 1e-3 * rng.random((n, n))
    for _ in range(20):
        W /= W.sum(1, keepdims=True)
        W /= W.sum(0, keepdims=True)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val, phases = fr.fram_assign(ctx, n, dev(torch, W), perm, with_phases=True)
    p = perm.cpu().numpy().astype(np.int64)
    ref = o.lap_max(W)
    assert abs(val - W[np.arange(n), ref].sum()) <= 1e-12 * n
    assert np.array_equal(p, ref)
    assert phases in (-1, 12)


def test_assign_one_column_preferred_runs_the_auction(torch_cuda, ctx):
    # Every row's maximum is column 7 and the rest differs by 1e-3 noise:
    # from the argmax start the completion needs more than its 64 n step
    # budget, so the epsilon-scaling auction runs and the completion
    # restarts from its prices.  The noise makes the optimum unique.
    torch = torch_cuda
    n = 1100
    rng = np.random.default_rng(12)
    b = rng.random(n)
    b[7] = 2.0
    W = b[None, :] + 1e-3 * rng.random((n, n))
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    _, val, phases = fr.fram_assign(ctx, n, dev(torch, W), perm, with_phases=True)
    p = perm.cpu().numpy().astype(np.int64)
    ref = o.lap_max(W)
    assert np.array_equal(p, ref)
    assert abs(val - W[np.arange(n), ref].sum()) <= 1e-12 * n
    assert phases == 12


# ------------------------------------------------------------ full solve
def solve_gpu(torch, ctx, g, params=None, K=None, host=False):
    n = g.n
    if host:
        A, B = g.A, g.B
        X = np.empty((n, n))
        P = np.empty(n, dtype=np.int32)
    else:
        A, B = dev(torch, g.A), dev(torch, g.B)
        X = torch.empty((n, n), dtype=torch.float64, device="cuda")
        P = torch.empty(n, dtype=torch.int32, device="cuda")
    Kd = None if K is None else (K if host else dev(torch, K))
    params = params or fr.fram_default_params(theta=g.theta)
    _, info = fr.fram_solve(ctx, n, A, B, Kd, params, X, P)
    if not host:
        X, P = X.cpu().numpy(), P.cpu().numpy()
    return X, P.astype(np.int64), info


def check_against_oracle(g, X, P, info, ref, rtol=RTOL_N):
    assert info.outer_iters == ref.outer_iters
    assert relF(X, ref.N) <= rtol
    assert np.array_equal(P, ref.perm)
    assert abs(info.objective - ref.objective) <= 1e-12 * max(1.0, abs(ref.objective))
    assert abs(info.match_error - ref.match_error) <= 1e-10 * max(1.0, ref.match_error)
    assert abs(info.delta - ref.delta) <= 1e-6 * ref.delta + 1e-15


@pytest.mark.parametrize("seed", range(4))
def test_solve_small_er_matches_oracle(torch_cuda, ctx, seed):
    g = fi.small_er_pair(seed)
    ref = o.fram(g.A, g.B, theta=g.theta)
    X, P, info = solve_gpu(torch_cuda, ctx, g)
    check_against_oracle(g, X, P, info, ref)
    assert info.total_sweeps == ref.total_sweeps
    assert o.accuracy(P, g.truth) == 1.0


@pytest.mark.parametrize("n,p,theta", [(1, 0.5, 10.0), (2, 1.0, 10.0), (5, 0.8, 2.0),
                                       (127, 0.1, 10.0), (200, 0.1, 10.0), (257, 0.3, 2.0)])
def test_solve_sizes_matches_oracle(torch_cuda, ctx, n, p, theta):
    g = fi.er_pair(n, p, noise=0.05, seed=n, theta=theta)
    if n == 1:
        g.A[:] = 1.0
        g.B[:] = 0.5
    ref = o.fram(g.A, g.B, theta=theta)
    X, P, info = solve_gpu(torch_cuda, ctx, g)
    check_against_oracle(g, X, P, info, ref)


def test_solve_gaussian_dense_matches_oracle(torch_cuda, ctx):
    g = fi.gaussian_pair(300, jitter=0.01, seed=2)
    ref = o.fram(g.A, g.B, theta=g.theta)
    X, P, info = solve_gpu(torch_cuda, ctx, g)
    check_against_oracle(g, X, P, info, ref)


def test_solve_gaussian_dense_diffuse_rounding(torch_cuda, ctx):
    # At theta = 2 the final N of a dense pair is diffuse: 163 of 400 rows
    # lose their argmax column to another row, so the rounding is decided by
    # the augmenting paths.  The permutation must still be the oracle's.
    g = fi.gaussian_pair(400, jitter=0.01, seed=1)
    ref = o.fram(g.A, g.B, theta=g.theta)
    X, P, info = solve_gpu(torch_cuda, ctx, g)
    check_against_oracle(g, X, P, info, ref)
    assert info.lap_augmentations >= 100


def test_solve_with_node_term(torch_cuda, ctx):
    g = fi.small_er_pair(1)
    rng = np.random.default_rng(2)
    F = rng.random((g.n, 4))
    Ft = np.empty_like(F)
    Ft[g.truth] = F
    K = F @ Ft.T
    ref = o.fram(g.A, g.B, K=K, theta=g.theta)
    X, P, info = solve_gpu(torch_cuda, ctx, g, K=K)
    check_against_oracle(g, X, P, info, ref)


def test_host_and_device_inputs_agree(torch_cuda, ctx):
    g = fi.small_er_pair(2)
    Xd, Pd, id_ = solve_gpu(torch_cuda, ctx, g)
    Xh, Ph, ih = solve_gpu(torch_cuda, ctx, g, host=True)
    assert np.array_equal(Xd, Xh) and np.array_equal(Pd, Ph)
    assert id_.objective == ih.objective


def test_solve_is_deterministic(torch_cuda, ctx):
    g = fi.er_pair(300, 0.1, noise=0.05, seed=9)
    X1, P1, _ = solve_gpu(torch_cuda, ctx, g)
    X2, P2, _ = solve_gpu(torch_cuda, ctx, g)
    assert np.array_equal(X1, X2) and np.array_equal(P1, P2)


def test_solve_rejects_invalid_and_degenerate(torch_cuda, ctx):
    torch = torch_cuda
    n = 8
    A = np.random.default_rng(0).random((n, n)); A = A + A.T
    P = np.empty(n, dtype=np.int32)
    bad = A.copy(); bad[0, 1] += 0.1                           # asymmetric
    st, _ = fr.fram_solve(ctx, n, bad, A, perm_out=P, check=False)
    assert st == fr.FRAM_ERR_INVALID and "symmetric" in fr.fram_last_error(ctx)
    neg = A.copy(); neg[2, 3] = neg[3, 2] = -1.0
    st, _ = fr.fram_solve(ctx, n, A, neg, perm_out=P, check=False)
    assert st == fr.FRAM_ERR_INVALID
    nan = A.copy(); nan[1, 1] = np.nan
    st, _ = fr.fram_solve(ctx, n, nan, A, perm_out=P, check=False)
    assert st == fr.FRAM_ERR_INVALID
    z = np.zeros((n, n))
    st, _ = fr.fram_solve(ctx, n, z, z, perm_out=P, check=False)
    assert st == fr.FRAM_ERR_DEGENERATE
    # edgeless first graph: gradient A N B is zero
    st, _ = fr.fram_solve(ctx, n, z, A, perm_out=P, check=False)
    assert st == fr.FRAM_ERR_DEGENERATE
    st, _ = fr.fram_solve(ctx, 0, A, A, perm_out=P, check=False)
    assert st == fr.FRAM_ERR_INVALID
    bad_p = fr.fram_default_params(alpha=0.0)
    st, _ = fr.fram_solve(ctx, n, A, A, params=bad_p, perm_out=P, check=False)
    assert st == fr.FRAM_ERR_INVALID
    # the context stays usable
    g = fi.small_er_pair(0)
    X, Pp, info = solve_gpu(torch, ctx, g)
    assert o.accuracy(Pp, g.truth) == 1.0


def test_solve_medium_full_size_matches_oracle(torch_cuda, ctx):
    # n = 1000 ER pair (p = 0.05, N(0,0.05) noise, 5% flips, theta = 10): the
    # benchmark's workload, whole N compared.
    g = fi.medium_er_pair(0)
    ref = o.fram(g.A, g.B, theta=g.theta)
    X, P, info = solve_gpu(torch_cuda, ctx, g)
    check_against_oracle(g, X, P, info, ref)
    assert info.total_sweeps == ref.total_sweeps


def test_device_wait_timeout_returns_error_and_context_survives(torch_cuda, ctx):
    # A grid barrier that can never complete (a flag nothing sets): the kernel
    # must leave through its time limit with FRAM_ERR_TIMEOUT, without a fault,
    # and the context must keep working afterwards.
    import time
    fr.fram_set_wait_limit(ctx, 200)
    try:
        t0 = time.perf_counter()
        st = fr.fram_selftest_wait_timeout(ctx, 4)
        dt = time.perf_counter() - t0
        assert st == fr.FRAM_ERR_TIMEOUT
        assert "wait" in fr.fram_last_error(ctx)
        assert 0.15 < dt < 5.0
    finally:
        fr.fram_set_wait_limit(ctx, 4000)
    g = fi.small_er_pair(0)
    X, P, info = solve_gpu(torch_cuda, ctx, g)
    assert o.accuracy(P, g.truth) == 1.0


@pytest.mark.parametrize("ns", [[30], [300], [30, 80], [30, 150, 300], [97, 97, 97, 50]])
def test_sdsn_grouped_equals_single(torch_cuda, ctx, ns):
    # The serving path's grouped SDSN: every problem on its solo sub-grid must
    # give exactly what fram_sdsn gives.
    torch = torch_cuda
    Xs = [dev(torch, np.random.default_rng(10 * k + n).random((n, n)) ** 2) for k, n in enumerate(ns)]
    Ds = [torch.empty_like(x) for x in Xs]
    _, sw, gm = fr.fram_sdsn_grouped(ctx, ns, Xs, Ds, 10.0, 1e-14, 200)
    for k, n in enumerate(ns):
        D1 = torch.empty_like(Xs[k])
        _, s1, g1 = fr.fram_sdsn(ctx, n, Xs[k], D1, 10.0, 1e-14, 200)
        assert sw[k] == s1 and gm[k] == g1
        assert torch.equal(Ds[k], D1)
