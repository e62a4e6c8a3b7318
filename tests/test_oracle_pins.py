"""Pins for the FP64 CPU oracle: each check compares the oracle against
something other than itself -- a closed form, an independent KKT or QP solve,
brute force over all permutations, scipy, or an invariant the paper proves.

Sections cited are those of arXiv 2508.00887.
"""
import itertools
import math
import os

import numpy as np
import pytest

import fram_inputs as fi
import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def rand_mat(n, seed, asym=True):
    rng = np.random.default_rng(seed)
    X = rng.random((n, n))
    if not asym:
        X = 0.5 * (X + X.T)
    return X


def constraint_matrix(n):
    """C y = 1 encodes Y 1 = 1 (rows) and Y^T 1 = 1 (columns) for y = vec_row(Y)."""
    C = np.zeros((2 * n, n * n))
    for i in range(n):
        C[i, i * n:(i + 1) * n] = 1.0
    for j in range(n):
        C[n + j, j::n] = 1.0
    return C


def kkt_affine_projection(X):
    """Textbook equality-constrained least squares: the minimum-norm correction
    y = x + C^T mu with C C^T mu = 1 - C x (solved by lstsq, C is rank 2n-1)."""
    n = X.shape[0]
    C = constraint_matrix(n)
    x = X.reshape(-1)
    mu = np.linalg.lstsq(C @ C.T, np.ones(2 * n) - C @ x, rcond=None)[0]
    return (x + C.T @ mu).reshape(n, n)


def dykstra_ds_projection(Z, iters=20000, tol=1e-15):
    """Exact Frobenius projection of Z onto D_n by Dykstra's algorithm
    (alternating projections with correction terms onto the affine set and the
    nonnegative orthant).  Uses the KKT affine projection above, not the oracle."""
    n = Z.shape[0]
    C = constraint_matrix(n)
    G = np.linalg.pinv(C @ C.T)

    def paff(Y):
        y = Y.reshape(-1)
        return (y + C.T @ (G @ (np.ones(2 * n) - C @ y))).reshape(n, n)

    X = Z.copy()
    P = np.zeros_like(Z)
    Q = np.zeros_like(Z)
    for _ in range(iters):
        Yk = paff(X + P)
        P = X + P - Yk
        Xn = np.maximum(Yk + Q, 0.0)
        Q = Yk + Q - Xn
        if np.max(np.abs(Xn - X)) < tol:
            X = Xn
            break
        X = Xn
    return X


def slsqp_fra(Xhat, theta):
    """Generic QP solve of the FRA problem (Thm. 1): max <D, Xhat> - <D, D>/theta
    over D_n, with scipy's SLSQP."""
    from scipy.optimize import minimize
    n = Xhat.shape[0]
    C = constraint_matrix(n)[:-1]               # drop one redundant row (rank 2n-1)
    x = Xhat.reshape(-1)
    fun = lambda d: -(d @ x) + (d @ d) / theta
    jac = lambda d: -x + 2.0 * d / theta
    cons = [{"type": "eq", "fun": lambda d: C @ d - 1.0, "jac": lambda d: C}]
    d0 = np.full(n * n, 1.0 / n)
    res = minimize(fun, d0, jac=jac, constraints=cons, bounds=[(0, None)] * (n * n),
                   method="SLSQP", options=dict(ftol=1e-15, maxiter=2000))
    return res.x.reshape(n, n)


def fra_value(D, Xhat, theta):
    return float(np.sum(D * Xhat) - np.sum(D * D) / theta)


def brute_lap(W):
    n = W.shape[0]
    best, arg = -math.inf, None
    for p in itertools.permutations(range(n)):
        v = sum(W[i, p[i]] for i in range(n))
        if v > best:
            best, arg = v, p
    return np.array(arg), best


def brute_qap(A, B):
    n = A.shape[0]
    best, arg = -math.inf, None
    for p in itertools.permutations(range(n)):
        p = np.array(p)
        v = o.objective(A, B, p)
        if v > best:
            best, arg = v, p
    return arg, best


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split("|")])
    return rows


# ------------------------------------------------- eq. 7: P1 and P2, Thm. 5
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("seed", [0, 1])
def test_p1_equals_kkt_least_squares(n, seed):
    X = rand_mat(n, seed) * 3.0 - 1.0          # asymmetric, mixed signs
    Y = o.p1(X)
    Yk = kkt_affine_projection(X)
    assert np.max(np.abs(Y - Yk)) < 1e-13
    assert np.max(np.abs(Y.sum(1) - 1)) < 1e-14 * max(n, 1) + 1e-15
    assert np.max(np.abs(Y.sum(0) - 1)) < 1e-14 * max(n, 1) + 1e-15


def test_p1_total_mass_is_n():
    # Appendix, SDSN convergence criterion: sum of P1(X) equals n.
    for n in (3, 17, 64):
        Y = o.p1(rand_mat(n, n) * 5)
        assert abs(Y.sum() - n) < 1e-12 * n


def test_p2_is_orthant_projection():
    X = rand_mat(5, 3) - 0.5
    assert np.array_equal(o.p2(X), (X + np.abs(X)) / 2)
    assert np.all(o.p2(X) >= 0)


def test_p3_lemma_is_zero_sum_projection():
    # Lemma of Thm. 7: P3 projects onto {Y1 = 0, Y^T 1 = 0}; check against KKT
    # with a zero right-hand side, built independently.
    n = 5
    X = rand_mat(n, 9) - 0.3
    C = constraint_matrix(n)
    x = X.reshape(-1)
    mu = np.linalg.lstsq(C @ C.T, -C @ x, rcond=None)[0]
    ref = (x + C.T @ mu).reshape(n, n)
    assert np.max(np.abs(o.p3(X) - ref)) < 1e-13


# ------------------------------------------------- golden worked examples
def test_sdsn_golden_2x2():
    for name, theta, gtol, ks, xs, sweeps, ds, g in read_golden("sdsn_2x2.txt"):
        X = np.array([float(v) for v in xs.split()]).reshape(2, 2)
        D = np.array([float(v) for v in ds.split()]).reshape(2, 2)
        r = o.sdsn(X, float(theta), float(gtol), int(ks))
        assert r.sweeps == int(sweeps), name
        assert np.array_equal(r.D, D), name
        assert r.gamma == float(g), name


# ------------------------------------------------- Alg. 2: SDSN vs the FRA QP
def test_sdsn_one_sweep_exact_when_p1_nonnegative():
    # If P1(theta/2 Xhat) >= 0, P2 is the identity and the first sweep already
    # lands on D_n at the exact projection, i.e. the FRA solution of Thm. 1.
    n, theta = 4, 0.2
    X = rand_mat(n, 5)
    Xhat = X / X.max()
    assert np.all(o.p1(theta / 2 * Xhat) >= 0)
    r = o.sdsn(X, theta, 1e-14, 200)
    assert r.sweeps == 1 and r.converged
    D_qp = slsqp_fra(Xhat, theta)
    D_dy = dykstra_ds_projection(theta / 2 * Xhat)
    assert np.max(np.abs(r.D - D_dy)) < 1e-12
    assert np.max(np.abs(r.D - D_qp)) < 1e-8


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sdsn_feasible_and_bounded_by_qp(seed):
    # In general SDSN is alternating projection (reading (iv)): its limit is a
    # feasible point, so its FRA value cannot exceed the QP optimum, which the
    # exact (Dykstra) projection attains.
    n, theta = 5, 10.0
    X = rand_mat(n, 100 + seed)
    Xhat = X / X.max()
    r = o.sdsn(X, theta, 1e-15, 100000)
    assert r.converged
    assert np.all(r.D >= 0)
    assert np.max(np.abs(r.D.sum(0) - 1)) < 1e-12 and np.max(np.abs(r.D.sum(1) - 1)) < 1e-12
    D_dy = dykstra_ds_projection(theta / 2 * Xhat)
    D_qp = slsqp_fra(Xhat, theta)
    v_sd, v_dy, v_qp = (fra_value(D, Xhat, theta) for D in (r.D, D_dy, D_qp))
    assert abs(v_dy - v_qp) < 1e-7
    assert v_sd <= v_dy + 1e-12


def test_sdsn_theta_to_zero_limit():
    # Thm. 4: D -> 11^T/n as theta -> 0, with a first-order deviation.
    n = 6
    X = rand_mat(n, 11)
    J = np.full((n, n), 1.0 / n)
    errs = []
    for theta in (1e-2, 1e-4, 1e-6):
        r = o.sdsn(X, theta, 1e-14, 200)
        assert r.sweeps == 1
        errs.append(np.max(np.abs(r.D - J)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6
    assert abs(errs[0] / errs[1] - 100) < 1e-6 * 100


def test_sdsn_theta_to_infinity_limit():
    # Cor. of Thm. 3: with a unique LAP optimum, D^theta tends to that
    # permutation.  The LAP optimum is found by brute force.
    n = 5
    X = rand_mat(n, 21)
    perm, _ = brute_lap(X)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1
    r = o.sdsn(X, 400.0, 1e-13, 400000)
    assert r.converged
    assert np.max(np.abs(r.D - P)) < 1e-6


def test_eps_bound_thm2():
    # Thm. 2: (<D_inf, X> - <D_theta, X>)/n <= 1/theta, D_inf from brute force.
    for seed in range(4):
        n = 5
        X = rand_mat(n, 40 + seed)
        Xhat = X / X.max()
        _, best = brute_lap(Xhat)
        for theta in (0.5, 2.0, 10.0):
            r = o.sdsn(X, theta, 1e-15, 200000)
            eps = (best - np.sum(r.D * Xhat)) / n
            assert eps <= 1.0 / theta + 1e-12


def test_sdsn_invariants_on_fram_iterate():
    # gamma >= 0 after a clamp and non-increasing (appendix); output >= 0;
    # on calls that converge at 1e-14, all row/col sums within 1e-12.
    g = fi.er_pair(120, 0.2, noise=0.02, seed=4)
    As, Bs, _, _ = o.prescale(g.A, g.B)
    N = o.initial_assignment(120, False)
    X = o.gradient(As, N, Bs)
    r = o.sdsn(X, 2.0, 1e-14, 20000, keep_history=True)
    assert r.converged
    assert np.all(r.D >= 0)
    h = np.array(r.gammas)
    assert np.all(h[:-1] >= -1e-15)
    assert np.all(np.diff(h) <= 1e-13)
    assert np.max(np.abs(r.D.sum(0) - 1)) < 1e-12 and np.max(np.abs(r.D.sum(1) - 1)) < 1e-12


def test_sdsn_degenerate_zero_input():
    with pytest.raises(o.DegenerateError):
        o.sdsn(np.zeros((3, 3)), 2.0)


# ------------------------------------------------- eq. 3: gradient of Phi
def test_gradient_is_derivative_of_objective():
    # Phi(N) = 1/2 <N^T A N, B> + lam <N, K>; for symmetric A, B its gradient is
    # A N B + lam K.  Central finite differences on random entries.
    n = 6
    rng = np.random.default_rng(3)
    A = rand_mat(n, 1, asym=False)
    B = rand_mat(n, 2, asym=False)
    K = rng.random((n, n))
    N = rng.random((n, n))

    def phi(M):
        return 0.5 * np.sum((M.T @ A @ M) * B) + 0.7 * np.sum(M * K)

    G = o.gradient(A, N, B, K, 0.7)
    h = 1e-6
    for (i, j) in [(0, 0), (1, 4), (5, 2), (3, 3)]:
        E = np.zeros((n, n))
        E[i, j] = h
        fd = (phi(N + E) - phi(N - E)) / (2 * h)
        assert abs(fd - G[i, j]) < 1e-7


def test_gradient_columns_equal_the_finite_difference_pinned_gradient():
    # The column form is the same X: checked against gradient() (pinned above
    # by finite differences) and against the written-out triple sum.
    n = 9
    rng = np.random.default_rng(5)
    A = rand_mat(n, 4, asym=False)
    B = rand_mat(n, 5, asym=False)
    K = rng.random((n, n))
    N = rng.random((n, n))
    cols = [0, 3, 8, 3]
    Xc = o.gradient_columns(A, N, B, cols, K, 0.7)
    assert np.allclose(Xc, o.gradient(A, N, B, K, 0.7)[:, cols], rtol=1e-14, atol=0)
    j = 8
    direct = [sum(A[i, k] * N[k, l] * B[l, j] for k in range(n) for l in range(n)) + 0.7 * K[i, j]
              for i in range(n)]
    assert np.allclose(Xc[:, 2], direct, rtol=1e-13, atol=0)


# ------------------------------------------------- Alg. 1 steps 7-8
def test_damped_update_delta_closed_form():
    # alpha = 1 from N = 11^T/n to D = I: ||I - J/n||_F^2 = n - 1, ||I||_F^2 = n.
    for n in (2, 7, 30):
        Nn, d = o.damped_update(np.full((n, n), 1.0 / n), np.eye(n), 1.0)
        assert np.array_equal(Nn, np.eye(n))
        assert abs(d - math.sqrt((n - 1) / n)) < 1e-15
    # alpha = 0 leaves N unchanged, delta = 0.
    N = rand_mat(4, 1)
    Nn, d = o.damped_update(N, rand_mat(4, 2), 0.0)
    assert np.array_equal(Nn, N) and d == 0.0


# ------------------------------------------------- eq. 2: the LAP
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_lap_equals_brute_force(n):
    for seed in range(4):
        W = rand_mat(n, 300 + seed + 10 * n)
        perm = o.lap_max(W)
        bperm, best = brute_lap(W)
        assert sorted(perm.tolist()) == list(range(n))
        assert abs(W[np.arange(n), perm].sum() - best) < 1e-12
        assert np.array_equal(perm, bperm)      # unique optimum for random W


@pytest.mark.parametrize("n", [10, 64, 257])
def test_lap_equals_scipy(n):
    from scipy.optimize import linear_sum_assignment
    for seed in range(2):
        W = rand_mat(n, 7 * n + seed)
        perm = o.lap_max(W)
        r, c = linear_sum_assignment(W, maximize=True)
        assert abs(W[np.arange(n), perm].sum() - W[r, c].sum()) < 1e-9
        assert np.array_equal(perm, c[np.argsort(r)])


def test_lap_ties_valid_and_optimal():
    # All-equal weights: every permutation is optimal; the oracle's tie rule
    # (first minimum) returns the identity.
    n = 6
    perm = o.lap_max(np.ones((n, n)))
    assert np.array_equal(perm, np.arange(n))
    W = np.kron(np.eye(3), np.ones((2, 2)))     # block ties
    perm = o.lap_max(W)
    assert abs(W[np.arange(6), perm].sum() - 6) < 1e-12


# ------------------------------------------------- eq. 1 and Sec. 7 criteria
def test_objective_gather_equals_dense_trace():
    n = 9
    A = rand_mat(n, 1, asym=False)
    B = rand_mat(n, 2, asym=False)
    K = rand_mat(n, 3)
    perm = np.random.default_rng(0).permutation(n)
    M = np.zeros((n, n))
    M[np.arange(n), perm] = 1
    dense = 0.5 * np.trace(M.T @ A @ M @ B.T) + 0.3 * np.trace(M.T @ K)
    assert abs(o.objective(A, B, perm, K, 0.3) - dense) < 1e-12
    # ||A - M B M^T||^2 = ||A||^2 + ||B||^2 - 4 Phi_edge (Sec. 7 criterion vs eq. 1)
    err = o.matching_error(A, B, perm)
    phi = o.objective(A, B, perm)
    assert abs((2 * err) ** 2 - (np.sum(A * A) + np.sum(B * B) - 4 * phi)) < 1e-10
    assert abs(err - 0.5 * np.linalg.norm(A - M @ B @ M.T)) < 1e-12


def test_accuracy_definition():
    assert o.accuracy(np.array([0, 1, 2, 3]), np.array([0, 1, 3, 2])) == 0.5
    assert o.accuracy(np.array([0, 1, 2]), np.array([0, -1, 1])) == 0.5


# ------------------------------------------------- Alg. 1 end to end
def test_fram_scale_invariance_bit_exact_and_general():
    g = fi.small_er_pair(3)
    r0 = o.fram(g.A, g.B, theta=g.theta)
    r4 = o.fram(16.0 * g.A, 16.0 * g.B, theta=g.theta)     # 4^2: sqrt(c) scales by 4
    assert np.array_equal(r0.N, r4.N) and np.array_equal(r0.perm, r4.perm)
    r3 = o.fram(3.7 * g.A, 3.7 * g.B, theta=g.theta)
    assert np.linalg.norm(r3.N - r0.N) / np.linalg.norm(r0.N) < 1e-13
    assert np.array_equal(r0.perm, r3.perm)


def test_fram_relabelling_equivariance():
    g = fi.small_er_pair(5)
    n = g.n
    rng = np.random.default_rng(77)
    q, s = rng.permutation(n), rng.permutation(n)
    Q = np.eye(n)[q]                    # (Q A Q^T)_ij = A[q_i, q_j]
    R = np.eye(n)[s]
    r0 = o.fram(g.A, g.B, theta=g.theta)
    r1 = o.fram(Q @ g.A @ Q.T, R @ g.B @ R.T, theta=g.theta)
    expect = Q @ r0.N @ R.T
    assert np.linalg.norm(r1.N - expect) / np.linalg.norm(expect) < 1e-12
    # node i of the relabelled first graph is q[i]; it maps to r0.perm[q[i]],
    # which is node s^-1(r0.perm[q[i]]) of the relabelled second graph.
    sinv = np.argsort(s)
    assert np.array_equal(r1.perm, sinv[r0.perm[q]])


@pytest.mark.parametrize("seed", range(10))
def test_fram_planted_recovery_noiseless(seed):
    g = fi.er_pair(50, 0.2, noise=0.0, seed=seed, theta=10.0)
    r = o.fram(g.A, g.B, theta=g.theta)
    assert np.array_equal(r.perm, g.truth)


@pytest.mark.parametrize("seed", range(3))
def test_fram_planted_recovery_small_noise(seed):
    g = fi.small_er_pair(seed)
    r = o.fram(g.A, g.B, theta=g.theta)
    assert o.accuracy(r.perm, g.truth) == 1.0


@pytest.mark.parametrize("seed", range(4))
def test_fram_bounded_by_brute_force_qap(seed):
    n = 7
    g = fi.er_pair(n, 0.6, noise=0.0, seed=1000 + seed, theta=10.0)
    r = o.fram(g.A, g.B, theta=g.theta)
    bperm, best = brute_qap(g.A, g.B)
    assert r.objective <= best + 1e-12
    # Noiseless planted pair with random weights: the planted map is the unique
    # QAP optimum (up to ties of equal value, checked by value).
    assert abs(o.objective(g.A, g.B, g.truth) - best) < 1e-12


def test_fram_node_attribute_term_and_zero_init():
    # With K the initial N is 0 (reading (i)); K = F F~^T with F~ = M^T F gives
    # a consistent node term.  The run must be well defined and recover truth.
    g = fi.small_er_pair(1)
    rng = np.random.default_rng(2)
    F = rng.random((g.n, 4))
    Ft = np.empty_like(F)
    Ft[g.truth] = F
    K = F @ Ft.T
    r = o.fram(g.A, g.B, K=K, theta=g.theta)
    assert o.accuracy(r.perm, g.truth) == 1.0
    r2 = o.fram(16 * g.A, 16 * g.B, K=256 * K, theta=g.theta)   # (wA, wB, w^2 K)
    assert np.array_equal(r.N, r2.N)


def test_node_affinity_brute_force_and_closed_forms():
    # K[i, j] = sum_k F[i, k] F~[j, k] written out; the total 1^T K 1 equals
    # (F^T 1) . (F~^T 1); with F~ = F it is a Gram matrix (symmetric PSD); and
    # the node term of eq. 1 at a permutation M is sum_i <F[i], F~[pi(i)]>.
    rng = np.random.default_rng(4)
    F, Ft = rng.random((5, 3)), rng.random((5, 3))
    K = o.node_affinity(F, Ft)
    for i in range(5):
        for j in range(5):
            assert K[i, j] == pytest.approx(sum(F[i, k] * Ft[j, k] for k in range(3)), rel=1e-15)
    F, Ft = rng.random((40, 17)), rng.random((40, 17))
    K = o.node_affinity(F, Ft)
    assert K.sum() == pytest.approx(F.sum(0) @ Ft.sum(0), rel=1e-13)
    G = o.node_affinity(F, F)
    assert np.array_equal(G, G.T) or np.max(np.abs(G - G.T)) < 1e-15
    assert np.linalg.eigvalsh(0.5 * (G + G.T)).min() > -1e-12
    perm = rng.permutation(40)
    Z = np.zeros((40, 40))
    assert o.objective(Z, Z, perm, K=K, lam=1.0) == pytest.approx(
        sum(F[i] @ Ft[perm[i]] for i in range(40)), rel=1e-13)
    with pytest.raises(o.InvalidInputError):
        o.node_affinity(F, Ft[:, :5])


def test_attributed_pair_node_term_helps():
    # Descriptor noise well below the descriptor spread: the node term lifts
    # the matching on a dense pair (Sec. 7 uses attributes on image graphs).
    g = fi.attributed_pair(120, d=32, seed=3)
    K = o.node_affinity(g.F, g.Ft)
    assert K.min() >= 0.0 and np.allclose(np.linalg.norm(g.F, axis=1), 1.0)
    r = o.fram(g.A, g.B, K=K, theta=2.0)
    r0 = o.fram(g.A, g.B, theta=2.0)
    assert o.accuracy(r.perm, g.truth) >= o.accuracy(r0.perm, g.truth)
    assert o.accuracy(r.perm, g.truth) >= 0.95


# ------------------------------------------------ exact FRA projection (step 6 variant)
def test_simplex_thresholds_against_bisection():
    # sum_j max(0, z_j - t) = 1 solved by bisection on the decreasing
    # piecewise-linear left side: an independent computation of t.
    rng = np.random.default_rng(5)
    Z = rng.normal(size=(20, 13)) * rng.choice([0.1, 1.0, 10.0], size=(20, 1))
    t = o.simplex_thresholds(Z)
    for i in range(Z.shape[0]):
        lo, hi = Z[i].max() - 1.0, Z[i].max()        # f(lo) >= 0 >= f(hi)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if np.maximum(0.0, Z[i] - mid).sum() >= 1.0:
                lo = mid
            else:
                hi = mid
        assert abs(t[i] - 0.5 * (lo + hi)) <= 1e-12 * max(1.0, abs(t[i]))
        assert abs(np.maximum(0.0, Z[i] - t[i]).sum() - 1.0) <= 1e-12


@pytest.mark.parametrize("n,theta,seed", [(6, 10.0, 0), (30, 10.0, 1), (30, 2.0, 2), (80, 10.0, 3)])
def test_fra_exact_kkt_certificate(n, theta, seed):
    # D = max(0, Y0 - a 1^T - 1 b^T) with unit row and column sums satisfies
    # the KKT conditions of the convex QP, so it is the projection; this
    # certificate does not depend on how a and b were found.
    X = rand_mat(n, 200 + seed)
    r = o.fra_exact(X, theta, tol=1e-12)
    assert r.converged and r.residual <= 1e-12
    Y0 = (theta / 2.0) * (X / X.max())
    assert np.array_equal(r.D, np.maximum(0.0, Y0 - r.a[:, None] - r.b[None, :]))
    assert np.all(r.D >= 0)
    assert np.max(np.abs(r.D.sum(1) - 1)) <= 1e-12 and np.max(np.abs(r.D.sum(0) - 1)) <= 1e-12


def test_fra_exact_equals_dykstra_and_qp():
    for seed in range(3):
        n, theta = 5, 10.0
        X = rand_mat(n, 300 + seed)
        Xhat = X / X.max()
        D = o.fra_exact(X, theta, tol=1e-14).D
        assert np.max(np.abs(D - dykstra_ds_projection(theta / 2 * Xhat))) < 1e-9
        D_qp = slsqp_fra(Xhat, theta)
        assert abs(fra_value(D, Xhat, theta) - fra_value(D_qp, Xhat, theta)) < 1e-7
        assert fra_value(D, Xhat, theta) >= fra_value(D_qp, Xhat, theta) - 1e-12


def test_fra_exact_is_p1_when_nothing_clamps():
    # Y0 large and flat enough that P1(Y0) >= 0: the affine projection is
    # already in D_n, so it is the exact projection (one SDSN sweep too).
    n, theta = 7, 10.0
    X = 1.0 + 0.01 * rand_mat(n, 7)
    Y0 = theta / 2 * X / X.max()
    P1 = kkt_affine_projection(Y0)
    assert np.all(P1 > 0)
    r = o.fra_exact(X, theta, tol=1e-14)
    assert np.max(np.abs(r.D - P1)) < 1e-12
    assert np.max(np.abs(o.sdsn(X, theta, 1e-14, 1).D - r.D)) < 1e-12


def test_fra_exact_limits_in_theta():
    # Thm. 4 (theta -> 0: 11^T/n) and Cor. of Thm. 3 (theta -> inf: the LAP
    # permutation, found by brute force).
    n = 5
    X = rand_mat(n, 21)
    assert np.max(np.abs(o.fra_exact(X, 1e-6).D - 1.0 / n)) < 1e-6
    perm, _ = brute_lap(X)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1
    assert np.max(np.abs(o.fra_exact(X, 1e4).D - P)) < 1e-9


def test_fra_exact_is_closest_feasible_point():
    # Every other doubly stochastic matrix is at least as far from Y0:
    # permutations, the centre, Sinkhorn-balanced matrices, converged SDSN.
    n, theta = 8, 10.0
    X = rand_mat(n, 9)
    Y0 = theta / 2 * X / X.max()
    d_star = np.linalg.norm(o.fra_exact(X, theta).D - Y0)
    rng = np.random.default_rng(1)
    cands = [np.full((n, n), 1.0 / n), o.sdsn(X, theta, 1e-15, 100000).D]
    for _ in range(20):
        P = np.eye(n)[rng.permutation(n)]
        cands.append(P)
        M = rng.random((n, n))
        for _ in range(200):
            M /= M.sum(1, keepdims=True)
            M /= M.sum(0, keepdims=True)
        cands.append(M)
    for D in cands:
        assert np.linalg.norm(D - Y0) >= d_star - 1e-12


def test_fra_exact_over_relaxation_reaches_the_same_point():
    X = rand_mat(40, 4)
    a = o.fra_exact(X, 10.0, tol=1e-12)
    b = o.fra_exact(X, 10.0, tol=1e-12, omega=1.6)
    assert np.max(np.abs(a.D - b.D)) < 1e-10


def test_fram_exact_projection_recovers_and_is_scale_invariant():
    g = fi.er_pair(40, 0.3, noise=0.0, seed=8, theta=10.0)
    r = o.fram(g.A, g.B, theta=10.0, projection="exact", omega=1.6)
    assert o.accuracy(r.perm, g.truth) == 1.0
    r4 = o.fram(4 * g.A, 4 * g.B, theta=10.0, projection="exact", omega=1.6)
    assert np.array_equal(r.N, r4.N) and r.outer_iters == r4.outer_iters


def test_validation_rejects_bad_inputs():
    A = rand_mat(4, 1, asym=False)
    with pytest.raises(o.InvalidInputError):
        o.fram(rand_mat(4, 1), A)                 # not symmetric
    with pytest.raises(o.InvalidInputError):
        o.fram(-A, A)                             # negative
    B = A.copy()
    B[0, 1] = B[1, 0] = np.nan
    with pytest.raises(o.InvalidInputError):
        o.fram(A, B)
    with pytest.raises(o.DegenerateError):
        o.fram(np.zeros((3, 3)), np.zeros((3, 3)))
