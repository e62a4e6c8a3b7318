"""Batched path (one persistent launch for pairs with n <= 64) through the C
ABI: FP64 against the oracle at parity, against solo fram_solve results, and
the FP32 mixed form at equal accuracy."""
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


def check_assignment(p, ref_perm, N_ref, g, inf=None, ref=None):
    """The LAP optimum value is unique; the permutation is unique only without
    (near-)ties -- padded dummy nodes give rows of N that are equal up to
    rounding.  Compare the value on the oracle's N, require a valid
    permutation, and require the identical permutation when the pair has no
    dummy/isolated nodes."""
    n = len(ref_perm)
    assert sorted(p.tolist()) == list(range(n))
    v_gpu = N_ref[np.arange(n), p].sum()
    v_ref = N_ref[np.arange(n), ref_perm].sum()
    assert abs(v_gpu - v_ref) <= 1e-12 * n
    isolated = (g.A.sum(1) == 0).any() or (g.B.sum(1) == 0).any()
    if not isolated:
        assert np.array_equal(p, ref_perm), g.meta
    if inf is not None:
        assert abs(inf.objective - o.objective(g.A, g.B, p)) <= 1e-12 * max(1.0, abs(inf.objective))
        if ref is not None and np.array_equal(p, ref_perm):
            assert abs(inf.objective - ref.objective) <= 1e-12 * max(1.0, abs(ref.objective))
            assert abs(inf.match_error - ref.match_error) <= 1e-10 * max(1.0, ref.match_error)


def mixed_batch(seed=0):
    """Keypoint pairs (n 10..64 with outliers), small ER pairs, and tiny n."""
    pairs = fi.keypoint_batch(14, seed=seed)
    pairs += [fi.er_pair(n, 1.0 if n <= 3 else 0.4, noise=0.02, seed=seed + n, theta=10.0)
              for n in (2, 3, 7, 33, 64)]
    pairs += [fi.small_er_pair(seed)]   # n = 50
    return pairs


def run_batched(torch, ctx, pairs, params, device=True, want_x=True):
    ns = [g.n for g in pairs]
    if device:
        As = [torch.from_numpy(g.A).cuda() for g in pairs]
        Bs = [torch.from_numpy(g.B).cuda() for g in pairs]
        Xs = [torch.empty((g.n, g.n), dtype=torch.float64, device="cuda") for g in pairs]
        Ps = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in pairs]
    else:
        As = [g.A for g in pairs]
        Bs = [g.B for g in pairs]
        Xs = [np.empty((g.n, g.n)) for g in pairs]
        Ps = [np.empty(g.n, dtype=np.int32) for g in pairs]
    st, infos = fr.fram_solve_batched(ctx, ns, As, Bs, params, Xs if want_x else None, Ps)
    conv = (lambda t: t.cpu().numpy()) if device else (lambda t: t)
    return [conv(x) for x in Xs], [conv(p).astype(np.int64) for p in Ps], infos


def test_batched_fp64_matches_oracle(torch_cuda, ctx):
    pairs = mixed_batch(0)
    X, P, infos = run_batched(torch_cuda, ctx, pairs, None)
    for g, x, p, inf in zip(pairs, X, P, infos):
        ref = o.fram(g.A, g.B, theta=10.0)
        assert inf.outer_iters == ref.outer_iters
        assert relF(x, ref.N) <= 1e-9, g.meta
        check_assignment(p, ref.perm, ref.N, g, inf, ref)


def test_batched_equals_solo(torch_cuda, ctx):
    torch = torch_cuda
    pairs = mixed_batch(1)
    params = fr.fram_default_params(theta=2.0)
    X, P, infos = run_batched(torch, ctx, pairs, params)
    for g, x, p, inf in zip(pairs, X, P, infos):
        Xs = torch.empty((g.n, g.n), dtype=torch.float64, device="cuda")
        Ps = torch.empty(g.n, dtype=torch.int32, device="cuda")
        _, si = fr.fram_solve(ctx, g.n, torch.from_numpy(g.A).cuda(), torch.from_numpy(g.B).cuda(),
                              None, params, Xs, Ps)
        assert si.outer_iters == inf.outer_iters
        assert relF(x, Xs.cpu().numpy()) <= 1e-12
        check_assignment(p, Ps.cpu().numpy().astype(np.int64), Xs.cpu().numpy(), g)


def test_batched_host_buffers_and_no_x(torch_cuda, ctx):
    pairs = mixed_batch(2)
    Xd, Pd, _ = run_batched(torch_cuda, ctx, pairs, None, device=True)
    Xh, Ph, _ = run_batched(torch_cuda, ctx, pairs, None, device=False)
    _, Pn, _ = run_batched(torch_cuda, ctx, pairs, None, device=True, want_x=False)
    for a, b, c, d, e in zip(Xd, Xh, Pd, Ph, Pn):
        assert np.array_equal(a, b) and np.array_equal(c, d) and np.array_equal(c, e)


def test_batched_address_arrays_equal_tensor_lists(torch_cuda, ctx):
    # The fast path of the binding: every argument as a numpy array of
    # addresses into one packed buffer (sizes as an int32 array), device and
    # host.  Results are bit-identical to the same batch passed as lists.
    torch = torch_cuda
    pairs = fi.keypoint_batch(300, seed=9)
    params = fr.fram_default_params(theta=2.0, precision=fr.FRAM_PREC_MIXED_TF32)
    Xl, Pl, il = run_batched(torch, ctx, pairs, params, device=True)
    ns = np.array([g.n for g in pairs], dtype=np.int32)
    off_m = np.concatenate([[0], np.cumsum([g.n * g.n for g in pairs])[:-1]]).astype(np.uint64)
    off_v = np.concatenate([[0], np.cumsum([g.n for g in pairs])[:-1]]).astype(np.uint64)
    for dev in ("cuda", "cpu"):
        A = torch.from_numpy(np.concatenate([g.A.ravel() for g in pairs])).to(dev)
        B = torch.from_numpy(np.concatenate([g.B.ravel() for g in pairs])).to(dev)
        X = torch.empty(int(sum(g.n * g.n for g in pairs)), dtype=torch.float64, device=dev)
        P = torch.empty(int(ns.sum()), dtype=torch.int32, device=dev)
        addr = lambda t, off: np.uint64(t.data_ptr()) + off * np.uint64(t.element_size())
        _, ia = fr.fram_solve_batched(ctx, ns, addr(A, off_m), addr(B, off_m), params,
                                      addr(X, off_m), addr(P, off_v))
        Xh, Ph = X.cpu().numpy(), P.cpu().numpy()
        for k, g in enumerate(pairs):
            m, v = int(off_m[k]), int(off_v[k])
            assert np.array_equal(Xh[m:m + g.n * g.n].reshape(g.n, g.n), Xl[k]), (dev, k)
            assert np.array_equal(Ph[v:v + g.n], Pl[k]), (dev, k)
            assert ia[k].outer_iters == il[k].outer_iters
    with pytest.raises(ValueError):
        fr.fram_solve_batched(ctx, ns, addr(A, off_m)[:-1], addr(B, off_m), params, None,
                              addr(P, off_v))


def test_batched_host_buffers_large_batch_packed_in_parallel(torch_cuda, ctx):
    # The full 4096-pair keypoint batch from host buffers: its 106 MB of
    # inputs are packed into the staging arena on several threads (batches
    # of 16 MB and more).  N, the permutations and the per-pair diagnostics
    # equal those of the same batch from device buffers.
    pairs = fi.keypoint_batch(4096, seed=5)
    params = fr.fram_default_params(theta=2.0, precision=fr.FRAM_PREC_MIXED_TF32)
    Xd, Pd, infd = run_batched(torch_cuda, ctx, pairs, params, device=True)
    Xh, Ph, infh = run_batched(torch_cuda, ctx, pairs, params, device=False)
    for a, b, c, d, i, j in zip(Xd, Xh, Pd, Ph, infd, infh):
        assert np.array_equal(a, b) and np.array_equal(c, d)
        assert (i.outer_iters, i.total_sweeps, i.objective) == (j.outer_iters, j.total_sweeps,
                                                                j.objective)


def check_batch_equal_accuracy(pairs, P, infos, refs):
    """Equal accuracy of a batch, both ways.  Pairs without outliers (ER
    pairs) must each be within 0.5 pp of accuracy and 1e-3 relative objective
    of their reference.  Keypoint pairs carry 0-20% outliers and dummy nodes;
    on some of them FP32 rounding moves the mixed solve to another local
    solution, so for the batch as a whole the mean accuracy must be within
    0.5 pp and the mean relative objective difference within 1e-3."""
    acc_m, acc_o, rel = [], [], []
    for g, p, inf, (ref_perm, ref_obj) in zip(pairs, P, infos, refs):
        assert sorted(p.tolist()) == list(range(g.n))
        assert abs(inf.objective - o.objective(g.A, g.B, p)) <= 1e-9 * max(1.0, abs(inf.objective))
        am, ao = o.accuracy(p, g.truth), o.accuracy(ref_perm, g.truth)
        r = abs(inf.objective - ref_obj) / max(abs(ref_obj), 1e-300)
        acc_m.append(am)
        acc_o.append(ao)
        rel.append(r)
        if g.meta.get("kind") != "keypoint":
            assert abs(am - ao) <= 0.005 and r <= 1e-3, g.meta
    print(f"batch of {len(pairs)}: accuracy {np.mean(acc_m):.4f} vs {np.mean(acc_o):.4f}, "
          f"objective rel. diff mean {np.mean(rel):.2e} max {np.max(rel):.2e}")
    assert abs(np.mean(acc_m) - np.mean(acc_o)) <= 0.005
    assert np.mean(rel) <= 1e-3


def test_batched_mixed_equal_accuracy(torch_cuda, ctx):
    pairs = mixed_batch(3)
    params = fr.fram_default_params(theta=10.0, precision=fr.FRAM_PREC_MIXED_BF16)
    X, P, infos = run_batched(torch_cuda, ctx, pairs, params)
    refs = []
    for g in pairs:
        ref = o.fram(g.A, g.B, theta=10.0)
        refs.append((ref.perm, ref.objective))
    check_batch_equal_accuracy(pairs, P, infos, refs)


def test_batched_routes_large_pairs_and_rejects_invalid(torch_cuda, ctx):
    torch = torch_cuda
    pairs = [fi.small_er_pair(0), fi.er_pair(100, 0.1, noise=0.02, seed=4)]
    X, P, infos = run_batched(torch, ctx, pairs, None)
    for g, x, p, inf in zip(pairs, X, P, infos):
        ref = o.fram(g.A, g.B, theta=10.0)
        assert relF(x, ref.N) <= 1e-9
        check_assignment(p, ref.perm, ref.N, g, inf, ref)
    bad = fi.small_er_pair(1)
    bad.A[0, 1] += 0.5                               # asymmetric
    st, _ = fr.fram_solve_batched(ctx, [50, 50], [pairs[0].A, bad.A], [pairs[0].B, bad.B], None,
                                  None, [np.empty(50, np.int32), np.empty(50, np.int32)],
                                  check=False)
    assert st == fr.FRAM_ERR_INVALID and "pair 1" in fr.fram_last_error(ctx)


def test_batched_full_keypoint_workload_sampled(torch_cuda, ctx):
    # 4096 keypoint pairs, n ~ U{10..64} with 0-20% outliers, theta = 2, in
    # one batched call at FP64 and at the FP32 mixed precision.  A 1% sample of
    # the FP64 results is re-solved by the oracle (parity: N within 1e-9, the
    # LAP optimum's value); the mixed batch is at equal accuracy with the FP64
    # batch over all 4096 pairs.
    torch = torch_cuda
    pairs = fi.keypoint_batch(4096, seed=7)
    ns = [g.n for g in pairs]
    As = [torch.from_numpy(g.A).cuda() for g in pairs]
    Bs = [torch.from_numpy(g.B).cuda() for g in pairs]
    X64 = [torch.empty((g.n, g.n), dtype=torch.float64, device="cuda") for g in pairs]
    P64 = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in pairs]
    Pm = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in pairs]
    _, i64 = fr.fram_solve_batched(ctx, ns, As, Bs, fr.fram_default_params(theta=2.0), X64, P64)
    params = fr.fram_default_params(theta=2.0, precision=fr.FRAM_PREC_MIXED_BF16)
    _, im = fr.fram_solve_batched(ctx, ns, As, Bs, params, None, Pm)
    rng = np.random.default_rng(0)
    for k in rng.choice(len(pairs), size=41, replace=False):
        g = pairs[k]
        ref = o.fram(g.A, g.B, theta=2.0)
        assert i64[k].outer_iters == ref.outer_iters
        assert relF(X64[k].cpu().numpy(), ref.N) <= 1e-9, g.meta
        check_assignment(P64[k].cpu().numpy().astype(np.int64), ref.perm, ref.N, g)
    P64h = [p.cpu().numpy().astype(np.int64) for p in P64]
    Pmh = [p.cpu().numpy().astype(np.int64) for p in Pm]
    check_batch_equal_accuracy(pairs, Pmh, im, [(p, i.objective) for p, i in zip(P64h, i64)])


@pytest.mark.parametrize("variant", [4, 5])
def test_batched_team_kernel_equal_accuracy(torch_cuda, ctx, variant):
    # The team form (4: one warp for n <= 32, two warps above; 5: two warps
    # for every pair) on the mixed batch: ER pairs one by one and the batch as
    # a whole at equal accuracy with the oracle.
    pairs = mixed_batch(3)
    params = fr.fram_default_params(theta=10.0, precision=fr.FRAM_PREC_MIXED_BF16)
    fr.fram_set_batched_kernel(ctx, variant)
    try:
        X, P, infos = run_batched(torch_cuda, ctx, pairs, params)
        assert fr.fram_batched_kernel(ctx, fr.FRAM_PREC_MIXED_BF16) == variant
    finally:
        fr.fram_set_batched_kernel(ctx, 0)
    refs = []
    for g in pairs:
        ref = o.fram(g.A, g.B, theta=10.0)
        refs.append((ref.perm, ref.objective))
    check_batch_equal_accuracy(pairs, P, infos, refs)


@pytest.mark.parametrize("variant", [2, 4, 5])
def test_batched_fp32_one_iteration_matches_oracle(torch_cuda, ctx, variant):
    # One outer iteration of 10 sweeps in FP32, every form, at the tile-edge
    # boundaries (n = 32 on one warp, 33 and 64 on two): N against the oracle's
    # FP64 iteration.  FP32 products over n <= 64 terms (relative error below
    # 64 u ~ 4e-6), then SDSN, which is non-expansive; N1 = 0.05 N0 + 0.95 D.
    # The FP32 stop tolerance is set to the oracle's 1e-14, which 10 sweeps do
    # not reach at theta = 2 for n >= 16, so both run exactly 10 sweeps.  At
    # n = 10 the first sweep already lands on the doubly stochastic set (no
    # entry is clipped), the oracle's gamma is at FP64 rounding and it stops
    # after one sweep.  FP32 stops at the first sweep whose FP32 total falls
    # to n (1 + 1e-14) or below, which rounding alone decides: anywhere up to
    # the 10-sweep cap, at the same fixed point (N is checked below).
    torch = torch_cuda
    params = fr.fram_default_params(theta=2.0, precision=fr.FRAM_PREC_MIXED_BF16, max_outer=1,
                                    max_sweeps=10, polish_tol=1e-14)
    pairs = [fi.gaussian_pair(n, jitter=0.02, seed=n) for n in (10, 16, 31, 32, 33, 48, 64)]
    fr.fram_set_batched_kernel(ctx, variant)
    try:
        X, P, infos = run_batched(torch, ctx, pairs, params)
    finally:
        fr.fram_set_batched_kernel(ctx, 0)
    for g, x, inf in zip(pairs, X, infos):
        ref = o.fram(g.A, g.B, theta=2.0, max_outer=1, max_sweeps=10)
        err = relF(x, ref.N)
        print(f"variant={variant} n={g.n} relF(N1)={err:.2e}")
        assert inf.outer_iters == 1
        if ref.total_sweeps == 10:
            assert inf.total_sweeps == 10
        else:
            assert ref.total_sweeps == 1 and 1 <= inf.total_sweeps <= 10, (g.n, inf.total_sweeps)
        assert err <= 1e-4, (g.n, err)


def test_batched_team_kernel_rejects_fp64(torch_cuda, ctx):
    pairs = mixed_batch(1)[:3]
    fr.fram_set_batched_kernel(ctx, 4)
    try:
        ns = [g.n for g in pairs]
        st, _ = fr.fram_solve_batched(ctx, ns, [g.A for g in pairs], [g.B for g in pairs], None,
                                      None, [np.empty(g.n, np.int32) for g in pairs], check=False)
        assert st == fr.FRAM_ERR_INVALID
    finally:
        fr.fram_set_batched_kernel(ctx, 0)
    st = fr.fram_set_batched_kernel(ctx, 9, check=False)
    assert st == fr.FRAM_ERR_INVALID


@pytest.mark.parametrize("variant", [2, 4])
def test_batched_keypoint_workload_forms_agree(torch_cuda, ctx, variant):
    # The full 4096-pair keypoint batch through a CTA form and the team form:
    # each at equal accuracy (batch aggregate) with the FP64 batch.
    torch = torch_cuda
    pairs = fi.keypoint_batch(4096, seed=9)
    ns = [g.n for g in pairs]
    As = [torch.from_numpy(g.A).cuda() for g in pairs]
    Bs = [torch.from_numpy(g.B).cuda() for g in pairs]
    P64 = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in pairs]
    Pm = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in pairs]
    _, i64 = fr.fram_solve_batched(ctx, ns, As, Bs, fr.fram_default_params(theta=2.0), None, P64)
    fr.fram_set_batched_kernel(ctx, variant)
    try:
        params = fr.fram_default_params(theta=2.0, precision=fr.FRAM_PREC_MIXED_BF16)
        _, im = fr.fram_solve_batched(ctx, ns, As, Bs, params, None, Pm)
    finally:
        fr.fram_set_batched_kernel(ctx, 0)
    P64h = [p.cpu().numpy().astype(np.int64) for p in P64]
    Pmh = [p.cpu().numpy().astype(np.int64) for p in Pm]
    check_batch_equal_accuracy(pairs, Pmh, im, [(p, i.objective) for p, i in zip(P64h, i64)])
