"""FP32 SDSN (Alg. 2 in the precision of Sec. 6's mixed-precision
architecture) against the FP64 oracle, step by step, through fram_sdsn_f32:
the kernel and launch configuration the mixed paths run inside fram_solve.

Covered variants (the grid and tile follow from n alone):
  * n = 1000, row stride 1024: 12 x 12 tiles of 84 x 84 held in shared
    memory for every sweep (the n = 1000 workload's configuration);
  * n = 2800, stride 2816: 234 x 236 tiles too large for shared memory, the
    sweep streams them through L2 (two 16-byte groups per lane);
  * n = 4039, stride 4096: the social workload's size, streamed, 64 MB
    iterate resident in L2 (six groups per lane);
  * n = 8192, stride 8192: the dense workload's size, 256 MB iterate
    streamed from HBM every sweep (six groups per lane);
  * small and ragged sizes: the warp forms (one warp for n <= 32, two for
    n <= 64, the boundaries on both sides), the one-CTA cluster form
    (n <= 256), odd n and unaligned strides.

Tolerance, derived from the arithmetic.  The oracle runs the same sweeps in
FP64 on the same (FP32-representable) input.  P1 (an affine projection) and
P2 (a projection onto a convex set) are both non-expansive in the Frobenius
norm, so an error present before a sweep is not amplified by it: after k
sweeps ||D32 - D64||_F is at most the sum of the rounding errors each sweep
adds.  Per element a sweep rounds y + a_i, then - b_j (a_i = 1/n + S/n^2 -
r_i/n, b_j = c_j/n), and a_i, b_j carry the FP32 rounding of 1/n, of the
products and of the row/column sums (at most 64 sequential additions deep
in every grid this library picks; 33 in the warp forms).  Summed in the Frobenius norm over the
matrix, sweep t adds at most
    u (2 ||Y_t|| + 3 sqrt(n) ||a_t|| + 2 sqrt(n) ||b_t||
       + 64 sqrt(n) (||r_t|| + ||c_t||) / n),          u = 2^-24,
and step 1 adds 2 u ||Y_0|| (the rounded scale and product).  `fp32_bound`
evaluates this on the oracle's own trajectory.  It is a worst case: the
measured distances are 50-200x smaller (2.5e-7 relative on skewed inputs,
1.2e-5 on the rank-1 first gradient at theta = 10, where a_i and b_j are
large next to the entries).  A structural slip (a dropped or mis-signed term,
a transposed or misplaced partial, a skipped sweep) gives O(1) errors.
gamma = S/n - 1: |gamma32 - gamma64| <= ||D32 - D64||_F (Cauchy-Schwarz over
n^2 entries, divided by n) plus the FP32 rounding of S, 64 u (1 + gamma).
The sweep count is fixed wherever D is compared, so that FP32 rounding
cannot move the stop by a sweep: gamma_tol = -1, below any gamma (gamma >= 0
after the clamp, up to rounding).  With gamma_tol = 0 a one-sweep-exact case
(n = 2) stops at gamma = -1e-16 in FP64 and one sweep later in FP32.
"""
import numpy as np
import pytest

import fram_inputs as fi
import oracle as o
import paper_2508_00887_gb300 as fr

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
SUM_DEPTH = 64
FIXED = -1.0  # a gamma_tol no sweep reaches


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


def fp32_bound(X, theta, sweeps):
    """First-order bound on ||D32 - D64||_F after `sweeps` sweeps (see the
    module docstring), evaluated along the oracle's trajectory."""
    n = X.shape[0]
    nrm = np.linalg.norm
    Y = (theta / 2.0) * (X / np.max(X))
    bound = 2 * U32 * nrm(Y)
    sq = np.sqrt(n)
    for _ in range(sweeps):
        r, c = Y.sum(1), Y.sum(0)
        a = 1.0 / n + r.sum() / n ** 2 - r / n
        b = c / n
        bound += U32 * (2 * nrm(Y) + 3 * sq * nrm(a) + 2 * sq * nrm(b)
                        + SUM_DEPTH * sq * (nrm(r) + nrm(c)) / n)
        Y = o.p2(o.p1(Y))
    return bound


def skewed_input(n, seed):
    """A nonnegative X with many near-zero entries (the clamp is active from
    the first sweep on), exactly representable in FP32."""
    X = np.random.default_rng(seed).random((n, n)) ** 3
    return X.astype(np.float32).astype(np.float64)


def gradient_input(n, seed):
    """The first FRAM gradient A N0 B of an ER pair (N0 = 11^T/n, reading (i)),
    rounded to FP32, as the mixed path hands it to SDSN."""
    g = fi.er_pair(n, 0.05, noise=0.05, flip_frac=0.05, seed=seed)
    As, Bs, _, _ = o.prescale(g.A, g.B)
    X = o.gradient(As, o.initial_assignment(n, False), Bs)
    return X.astype(np.float32).astype(np.float64)


def run_f32(torch, ctx, X, ld, theta, gamma_tol, sweeps, in_place=False, pad_value=7.0):
    """Run fram_sdsn_f32 on X stored with row stride ld; returns D (n x n,
    float64), the padding columns of the output buffer, sweeps and gamma."""
    n = X.shape[0]
    Xp = np.full((n, ld), pad_value, dtype=np.float32)
    Xp[:, :n] = X
    Xd = torch.from_numpy(Xp).cuda()
    Dd = Xd if in_place else torch.full((n, ld), pad_value, dtype=torch.float32, device="cuda")
    _, k, g = fr.fram_sdsn_f32(ctx, n, Xd, Dd, theta, gamma_tol, sweeps, ldx=ld, ldd=ld)
    Dh = Dd.cpu().numpy()
    return Dh[:, :n].astype(np.float64), Dh[:, n:], k, g


CASES = [
    # n, row stride, sweeps, theta, input
    (1000, 1024, 10, 10.0, "gradient"),
    (1000, 1000, 10, 2.0, "skewed"),
    (2800, 2816, 8, 10.0, "skewed"),
    (4039, 4096, 8, 10.0, "skewed"),
    (8192, 8192, 4, 2.0, "skewed"),
    (2, 2, 10, 2.0, "skewed"),
    (10, 13, 10, 10.0, "skewed"),
    (31, 31, 12, 2.0, "skewed"),
    (32, 36, 10, 10.0, "gradient"),
    (33, 33, 10, 2.0, "skewed"),
    (50, 50, 10, 10.0, "gradient"),
    (64, 64, 10, 10.0, "gradient"),
    (65, 67, 10, 2.0, "skewed"),
    (97, 101, 10, 2.0, "skewed"),
    (333, 333, 10, 10.0, "skewed"),
]


@pytest.mark.parametrize("n,ld,sweeps,theta,kind", CASES)
def test_sdsn_f32_matches_oracle(torch_cuda, ctx, n, ld, sweeps, theta, kind):
    X = gradient_input(n, 3) if kind == "gradient" else skewed_input(n, n + ld)
    ref = o.sdsn(X, theta, FIXED, sweeps)
    D, pad, k, g = run_f32(torch_cuda, ctx, X, ld, theta, FIXED, sweeps)
    dist = float(np.linalg.norm(D - ref.D))
    bound = fp32_bound(X, theta, sweeps)
    print(f"n={n} ld={ld} sweeps={k} relF={dist / np.linalg.norm(ref.D):.3e} "
          f"bound/dist={bound / max(dist, 1e-300):.1f} gamma={g:.6e} oracle={ref.gamma:.6e}")
    assert k == ref.sweeps == sweeps
    assert dist <= bound
    s_tol = SUM_DEPTH * U32 * (1.0 + abs(ref.gamma))
    assert abs(g - ref.gamma) <= bound + s_tol
    assert np.all(D >= 0.0)
    # gamma is the one of the returned matrix, and the padding is untouched
    assert abs((D.sum() / n - 1.0) - g) <= s_tol
    assert pad.size == 0 or np.all(pad == 7.0)


@pytest.mark.parametrize("n,ld", [(1000, 1024), (4039, 4096)])
def test_sdsn_f32_in_place_equals_out_of_place(torch_cuda, ctx, n, ld):
    # The mixed path runs SDSN in place on the gradient buffer.
    X = skewed_input(n, 11)
    D1, _, k1, g1 = run_f32(torch_cuda, ctx, X, ld, 10.0, 0.0, 6)
    D2, pad, k2, g2 = run_f32(torch_cuda, ctx, X, ld, 10.0, 0.0, 6, in_place=True)
    assert k1 == k2 == 6 and g1 == g2
    assert np.array_equal(D1, D2)
    assert np.all(pad == 7.0)


@pytest.mark.parametrize("n", [24, 40, 200])
def test_sdsn_f32_stops_at_gamma_tol(torch_cuda, ctx, n):
    # theta = 2 on a small dense input converges: the FP32 run stops at its
    # first sweep k with gamma32 <= tol.  gamma32 is within eps of the exact
    # gamma of that sweep (eps: the D bound plus the FP32 rounding of S, as in
    # the module docstring), so the exact gamma at the FP32 stop is at most
    # tol + eps, and every earlier sweep's exact gamma is above tol - eps.
    # n = 24 and 40 run the warp forms, n = 200 the one-CTA cluster.
    X = skewed_input(n, 5)
    tol = 1e-6
    ref = o.sdsn(X, 2.0, FIXED, 2000, keep_history=True)
    D, _, k, g = run_f32(torch_cuda, ctx, X, n, 2.0, tol, 2000)
    hist = np.array(ref.gammas)
    eps = fp32_bound(X, 2.0, k) + SUM_DEPTH * U32 * (1.0 + tol)
    assert g <= tol and 1 <= k < 2000
    assert hist[k - 1] <= tol + eps
    assert np.all(hist[:k - 1] > tol - eps)
    r, c = D.sum(1), D.sum(0)
    assert np.max(np.abs(r - 1)) <= n * (tol + eps) and np.max(np.abs(c - 1)) <= n * (tol + eps)


def test_sdsn_f32_rejects_bad_arguments(torch_cuda, ctx):
    torch = torch_cuda
    n = 64
    X = torch.rand((n, n), dtype=torch.float32, device="cuda")
    D = torch.empty_like(X)
    st, _, _ = fr.fram_sdsn_f32(ctx, n, X, D, 2.0, 0.0, 5, ldx=n - 1, check=False)
    assert st == fr.FRAM_ERR_INVALID
    st, _, _ = fr.fram_sdsn_f32(ctx, n, X.cpu(), D, 2.0, 0.0, 5, check=False)
    assert st == fr.FRAM_ERR_INVALID
    Z = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    st, _, _ = fr.fram_sdsn_f32(ctx, n, Z, D, 2.0, 0.0, 5, check=False)
    assert st == fr.FRAM_ERR_DEGENERATE
