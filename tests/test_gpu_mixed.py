"""Mixed-precision path (BF16/TF32 tensor-core gradient, FP32 SDSN with FP64
polish, FP64 update) through the C ABI.

Two kinds of checks:
 * the tensor-core GEMMs against a CPU emulation of the same rounding
   (operands rounded to BF16/TF32, T rounded after the first product, FP64
   sums): they differ only by FP32 accumulation order;
 * full solves against the FP64 oracle at "equal accuracy": planted-match
   accuracy within 0.5 percentage points and objective within 1e-3 relative
   (the mixed results also report the relative error of N).
"""
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


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def round_bf16(torch, x):
    return torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()


def round_tf32(x):
    """Round to nearest TF32 (10 mantissa bits), ties away from zero."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("precision", [fr.FRAM_PREC_MIXED_BF16, fr.FRAM_PREC_MIXED_TF32])
@pytest.mark.parametrize("n", [50, 128, 200, 300, 1000, 1500, 2048])
def test_gradient_lowp_matches_emulation(torch_cuda, ctx, precision, n):
    # Tile shapes: 128 x 64 up to ld = 1536 (n = 50 .. 1500), 128 x 128 at
    # ld = 2048.
    torch = torch_cuda
    rng = np.random.default_rng(n + 10 * precision)
    A = rng.random((n, n)); A = 0.5 * (A + A.T)
    B = rng.random((n, n)); B = 0.5 * (B + B.T)
    N = rng.random((n, n)) / n
    K = rng.random((n, n))
    rnd = (lambda x: round_bf16(torch, x)) if precision == fr.FRAM_PREC_MIXED_BF16 else round_tf32
    T = rnd(rnd(A) @ rnd(N))
    ref = T @ rnd(B) + 0.5 * K
    X = torch.empty((n, n), dtype=torch.float32, device="cuda")
    dev = lambda a: torch.from_numpy(a).cuda()
    fr.fram_gradient_lowp(ctx, n, dev(A), dev(N), dev(B), X, precision, dev(K), 0.5)
    Xg = X.cpu().numpy().astype(np.float64)
    # FP32 accumulation over n terms; T is re-rounded, so allow a few ulps of
    # the input format where a rounding boundary of T falls differently.  The
    # tensor cores' FP32 accumulation also drops low-order bits on each add:
    # a bias toward zero that grows linearly with the number of terms
    # (measured 2.0e-5 relative at n = 1500 and 2.7e-5 at n = 2048, about
    # 1.3e-8 n), so the TF32 bound grows with n, 1.5x above those values.
    tol = 2e-5 * max(1.0, n / 1000) if precision == fr.FRAM_PREC_MIXED_TF32 else 4e-4
    assert relF(Xg, ref) < tol
    exact = A @ N @ B + 0.5 * K
    assert relF(Xg, exact) < (2e-3 if precision == fr.FRAM_PREC_MIXED_TF32 else 1e-2)


def solve(torch, ctx, g, precision, max_polish=4):
    n = g.n
    A = torch.from_numpy(g.A).cuda()
    B = torch.from_numpy(g.B).cuda()
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    params = fr.fram_default_params(theta=g.theta, precision=precision, max_polish=max_polish)
    _, info = fr.fram_solve(ctx, n, A, B, None, params, X, P)
    return X.cpu().numpy(), P.cpu().numpy().astype(np.int64), info


# Relative Frobenius distance of the mixed N from the oracle's N allowed per
# precision: a few times the largest value measured on the workloads below
# (n = 50 to 1000 ER pairs, n = 300 Gaussian pair).  The gradient's input
# rounding (2^-9 relative for BF16, 2^-12 for TF32) sets its scale.
X_TOL = {fr.FRAM_PREC_MIXED_BF16: 5e-3, fr.FRAM_PREC_MIXED_TF32: 1e-3}


def check_equal_accuracy(g, ref, X, P, info):
    """Equal accuracy as the metric defines it, both ways: planted-match
    accuracy within 0.5 percentage points of the oracle's and objective within
    1e-3 relative of the oracle's (a mixed result that drifts to a different,
    better-scoring permutation fails too)."""
    acc_o = o.accuracy(ref.perm, g.truth)
    acc_m = o.accuracy(P, g.truth)
    assert abs(acc_m - acc_o) <= 0.005
    assert abs(info.objective - ref.objective) <= 1e-3 * abs(ref.objective)
    assert sorted(P.tolist()) == list(range(g.n))
    # the objective the kernels report is the one of the returned permutation
    assert abs(info.objective - o.objective(g.A, g.B, P)) <= 1e-9 * abs(info.objective)
    return relF(X, ref.N)


@pytest.mark.parametrize("precision", [fr.FRAM_PREC_MIXED_BF16, fr.FRAM_PREC_MIXED_TF32])
@pytest.mark.parametrize("seed", range(3))
def test_mixed_small_er_equal_accuracy(torch_cuda, ctx, precision, seed):
    g = fi.small_er_pair(seed)
    ref = o.fram(g.A, g.B, theta=g.theta)
    X, P, info = solve(torch_cuda, ctx, g, precision)
    err = check_equal_accuracy(g, ref, X, P, info)
    print(f"n={g.n} precision={precision} relF(N)={err:.3e}")
    assert err <= X_TOL[precision]
    assert info.total_sweeps > 0 and info.outer_iters >= 1


@pytest.mark.parametrize("precision", [fr.FRAM_PREC_MIXED_BF16, fr.FRAM_PREC_MIXED_TF32])
def test_mixed_medium_equal_accuracy(torch_cuda, ctx, precision):
    g = fi.medium_er_pair(0)
    ref = o.fram(g.A, g.B, theta=g.theta)
    X, P, info = solve(torch_cuda, ctx, g, precision)
    err = check_equal_accuracy(g, ref, X, P, info)
    print(f"precision={precision} relF(N)={err:.3e} outer={info.outer_iters} "
          f"sweeps={info.total_sweeps} polish={info.polish_sweeps}")
    assert err <= X_TOL[precision]


def test_mixed_dense_gaussian_equal_accuracy(torch_cuda, ctx):
    g = fi.gaussian_pair(300, jitter=0.01, seed=2)
    ref = o.fram(g.A, g.B, theta=g.theta)
    X, P, info = solve(torch_cuda, ctx, g, fr.FRAM_PREC_MIXED_BF16)
    err = check_equal_accuracy(g, ref, X, P, info)
    print(f"gaussian n={g.n} relF(N)={err:.3e}")
    assert err <= X_TOL[fr.FRAM_PREC_MIXED_BF16]


@pytest.mark.parametrize("n", [24, 40, 120])
def test_mixed_polish_reaches_fp64_tolerance(torch_cuda, ctx, n):
    # theta = 2 on a small dense pair, where SDSN converges.  (1) The FP32
    # phase reaches polish_tol, so the gate skips the FP64 polish.  (2) With
    # the FP32 phase capped at 3 sweeps, gamma is still large, the polish runs
    # and takes gamma to gamma_tol in FP64.  n = 24 and 40 run the polish in
    # its warp forms (one CTA of 2 or 4 warps), n = 120 in the grid form.
    torch = torch_cuda
    g = fi.gaussian_pair(n, jitter=0.01, seed=4)
    n = g.n
    A = torch.from_numpy(g.A).cuda()
    B = torch.from_numpy(g.B).cuda()
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    p = fr.fram_default_params(theta=2.0, precision=fr.FRAM_PREC_MIXED_BF16, max_polish=2000,
                               polish_tol=1e-6, max_sweeps=4000, max_outer=3)
    _, info = fr.fram_solve(ctx, n, A, B, None, p, None, P)
    assert info.polish_sweeps == 0
    p.max_sweeps = 2003                    # FP32 phase: at most 3 sweeps
    _, info = fr.fram_solve(ctx, n, A, B, None, p, None, P)
    assert info.polish_sweeps > 0
    assert info.gamma <= 1e-14 and info.sdsn_converged_last == 1


def test_mixed_stops_at_rounding_floor(torch_cuda, ctx):
    # BF16 gradients put a floor under delta (about 1e-4 at n = 1000), far
    # above delta_tol = 1e-6: the mixed paths stop at mixed_delta_tol or, if
    # delta stalls just above it, by the stall safeguard; with
    # mixed_delta_tol disabled the safeguard stops the loop once delta stops
    # contracting; with both disabled the loop runs to the cap.
    torch = torch_cuda
    g = fi.medium_er_pair(0)
    n = g.n
    A = torch.from_numpy(g.A).cuda()
    B = torch.from_numpy(g.B).cuda()
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    p = fr.fram_default_params(theta=g.theta, precision=fr.FRAM_PREC_MIXED_BF16, max_polish=4,
                               max_outer=60)
    _, info = fr.fram_solve(ctx, n, A, B, None, p, None, P)
    # stopped by one of the two floor rules of reading (ix), long before the cap
    assert info.outer_iters < 20
    assert info.delta <= p.mixed_delta_tol or info.delta <= p.stall_below
    assert o.accuracy(P.cpu().numpy(), g.truth) == 1.0
    p.mixed_delta_tol = 0.0
    _, info = fr.fram_solve(ctx, n, A, B, None, p, None, P)
    assert info.outer_iters < 60 and info.delta <= p.stall_below
    p.stall_ratio = 0.0
    _, info = fr.fram_solve(ctx, n, A, B, None, p, None, P)
    assert info.outer_iters == 60


def test_fp64_streaming_sizes_match_oracle(torch_cuda, ctx):
    # n = 2800: SDSN tiles of 234 x 236 (FP64 or FP32) exceed shared memory and
    # stream through L2 each sweep.  Two outer iterations of 50 sweeps of the
    # FP64 path against the oracle at the parity tolerance; the full mixed
    # solves of the same pair are compared with this path below.
    torch = torch_cuda
    g = fi.er_pair(2800, 0.05, noise=0.05, flip_frac=0.05, seed=3)
    ref = o.fram(g.A, g.B, theta=g.theta, max_outer=2, max_sweeps=50)
    n = g.n
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    p64 = fr.fram_default_params(theta=g.theta, max_outer=2, max_sweeps=50)
    _, info = fr.fram_solve(ctx, n, torch.from_numpy(g.A).cuda(), torch.from_numpy(g.B).cuda(),
                            None, p64, X, P)
    assert relF(X.cpu().numpy(), ref.N) <= 1e-9
    assert info.total_sweeps == ref.total_sweeps and info.outer_iters == 2
    assert abs(info.delta - ref.delta) <= 1e-9 * ref.delta


_FP64_SOLVES = {}


def fp64_solve(torch, ctx, n, seed):
    """An ER pair (p = 0.05, noise 0.05, 5% flips, theta = 10) of size n solved
    by the GPU FP64 path (which matches the oracle at the parity tolerance)."""
    if n not in _FP64_SOLVES:
        g = fi.er_pair(n, 0.05, noise=0.05, flip_frac=0.05, seed=seed)
        A = torch.from_numpy(g.A).cuda()
        B = torch.from_numpy(g.B).cuda()
        X = torch.empty((n, n), dtype=torch.float64, device="cuda")
        P = torch.empty(n, dtype=torch.int32, device="cuda")
        _, info = fr.fram_solve(ctx, n, A, B, None, fr.fram_default_params(theta=g.theta), X, P)
        _FP64_SOLVES[n] = (g, A, B, X.cpu().numpy(), P.cpu().numpy().astype(np.int64), info)
    return _FP64_SOLVES[n]


@pytest.mark.parametrize("precision", [fr.FRAM_PREC_MIXED_BF16, fr.FRAM_PREC_MIXED_TF32])
@pytest.mark.parametrize("n,seed", [(2800, 3), (4096, 4)])
def test_mixed_full_solve_streaming_equal_accuracy(torch_cuda, ctx, precision, n, seed):
    # Full mixed solves where the FP32 SDSN streams its tiles through L2 (n =
    # 2800: two 16-byte groups per lane; n = 4096: six) against the FP64 solve
    # of the same pair: equal accuracy both ways and N within the precision's
    # tolerance.
    torch = torch_cuda
    g, A, B, N64, P64, i64 = fp64_solve(torch, ctx, n, seed)
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    p = fr.fram_default_params(theta=g.theta, precision=precision, max_polish=4)
    _, info = fr.fram_solve(ctx, n, A, B, None, p, X, P)
    Pm = P.cpu().numpy().astype(np.int64)
    err = relF(X.cpu().numpy(), N64)
    acc_m, acc_64 = o.accuracy(Pm, g.truth), o.accuracy(P64, g.truth)
    print(f"n={n} precision={precision} relF(N)={err:.3e} acc={acc_m:.4f}/{acc_64:.4f} "
          f"obj={info.objective:.6f}/{i64.objective:.6f} outer={info.outer_iters}/{i64.outer_iters}")
    assert sorted(Pm.tolist()) == list(range(n))
    assert abs(acc_m - acc_64) <= 0.005
    assert abs(info.objective - i64.objective) <= 1e-3 * abs(i64.objective)
    assert err <= X_TOL[precision]
