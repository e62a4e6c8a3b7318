"""Plain, slow, FP64 CPU oracle of FRAM (Frobenius-Regularized Assignment
Matching, arXiv 2508.00887).

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg
and ``--impl reference``) may import it.  It shares no code with the CUDA
library and imports nothing from the product package.

Every function follows one passage of the paper, cited in its docstring, in
the paper's order and notation.  Matrix products use ``numpy.matmul`` (a
library primitive); everything else is written out.  Where the paper is
silent, garbled or inconsistent, the reading taken is stated where it is
used, as "Reading (x)".

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, KKT solves, brute force,
scipy, invariants).  The exact value of N after a capped SDSN on large inputs
has no closed form; there the oracle itself is the reference.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Default parameters: theta/lambda/alpha from Sec. 7 "Setting"; tolerances and
# caps are readings (ii)/(iii) because the paper gives none.
DEFAULTS = dict(lam=1.0, alpha=0.95, theta=10.0, delta_tol=1e-6, max_outer=100,
                gamma_tol=1e-14, max_sweeps=200)


class DegenerateError(ValueError):
    """max(X) <= 0 in SDSN step 1: X/max(X) is undefined (e.g. edgeless graphs)."""


class InvalidInputError(ValueError):
    """Input violates the graph model of Sec. 3 (square, symmetric, >= 0, finite)."""


# --------------------------------------------------------------------------
# Sec. 3 "Graph": input contract.  Reading (vii): A and A~ must be symmetric,
# nonnegative and finite; the gradient A N A~ is only grad(Phi) for symmetric
# inputs (eq. 3).
# --------------------------------------------------------------------------
def validate(A, B, K=None, sym_tol=1e-12):
    for name, M in (("A", A), ("B", B)) + ((("K", K),) if K is not None else ()):
        M = np.asarray(M)
        if M.ndim != 2 or M.shape[0] != M.shape[1]:
            raise InvalidInputError(f"{name} must be square")
        if not np.all(np.isfinite(M)):
            raise InvalidInputError(f"{name} has non-finite entries")
        if np.any(M < 0):
            raise InvalidInputError(f"{name} has negative entries")
    n = A.shape[0]
    if n < 1 or B.shape != A.shape or (K is not None and K.shape != A.shape):
        raise InvalidInputError("A, B (and K) must have the same shape n x n, n >= 1")
    for name, M in (("A", A), ("B", B)):
        mx = float(np.max(np.abs(M))) if M.size else 0.0
        if np.max(np.abs(M - M.T)) > sym_tol * max(mx, 1.0):
            raise InvalidInputError(f"{name} is not symmetric")


# --------------------------------------------------------------------------
# Alg. 1, steps 2-3: c = max(A, A~, K); A/sqrt(c), A~/sqrt(c), K/c (FP64).
# --------------------------------------------------------------------------
def prescale(A, B, K=None):
    c = max(float(np.max(A)), float(np.max(B)))
    if K is not None:
        c = max(c, float(np.max(K)))
    if c <= 0:
        raise DegenerateError("all inputs are zero")
    s = math.sqrt(c)
    return A / s, B / s, (K / c if K is not None else None), c


# --------------------------------------------------------------------------
# Alg. 1, step 1.  The paper writes X^(0) = 0 for the variable that the loop
# reads as N^(t-1).  Reading (i): N^(0) = 0 when K is given; N^(0) = 11^T/n
# (the centre of D_n, the theta -> 0 limit of Thm. 4) when K is absent, since
# otherwise X^(1) = 0 and X/max(X) in Alg. 2 step 1 is undefined.
# --------------------------------------------------------------------------
def initial_assignment(n, has_K):
    if has_K:
        return np.zeros((n, n))
    return np.full((n, n), 1.0 / n)


# --------------------------------------------------------------------------
# Eq. 1 node term <N, F F~^T> (Sec. 3 "Matching matrix"; its gradient is the
# lambda F F~^T of eq. 3): K[i, j] = <F[i], F~[j]>, node i of G against node
# j of G~.
# --------------------------------------------------------------------------
def node_affinity(F, Ft):
    F = np.asarray(F, dtype=np.float64)
    Ft = np.asarray(Ft, dtype=np.float64)
    if F.ndim != 2 or Ft.ndim != 2 or F.shape != Ft.shape or F.shape[0] < 1 or F.shape[1] < 1:
        raise InvalidInputError("F and F~ must both be n x d with n, d >= 1")
    return F @ Ft.T


# --------------------------------------------------------------------------
# Eq. 3 / Alg. 1 step 5: the QAP gradient  X = A N A~ + lambda K.
# --------------------------------------------------------------------------
def gradient(A, N, B, K=None, lam=1.0):
    X = (A @ N) @ B
    if K is not None:
        X = X + lam * K
    return X


def gradient_columns(A, N, B, cols, K=None, lam=1.0):
    """Columns `cols` of the same X (eq. 3), each as A (N B[:, j]) + lambda
    K[:, j]: two matrix-vector products per column, for sampled checks at
    sizes where the full n^3 product is too slow on the CPU."""
    cols = np.asarray(cols, dtype=np.int64)
    X = A @ (N @ B[:, cols])
    if K is not None:
        X = X + lam * K[:, cols]
    return X


# --------------------------------------------------------------------------
# Eq. 7: the two projections that SDSN alternates.
#   P1(X) = X + (I/n + (1^T X 1/n^2) I - X/n) 1 1^T - 1 1^T X / n
# Reading (v): the bracket mixes a matrix into a vector slot; taken
# elementwise it is  P1(X)_ij = X_ij + 1/n + S/n^2 - r_i/n - c_j/n  with
# S = 1^T X 1, r = X 1 (row sums), c = X^T 1 (column sums).  Thm. 5: this is
# the Frobenius projection onto {Y1 = 1, Y^T 1 = 1} for any square X.
#   P2(X) = (X + |X|)/2 = max(0, X).
# --------------------------------------------------------------------------
def p1(X):
    n = X.shape[0]
    S = np.sum(X)
    r = np.sum(X, axis=1)
    c = np.sum(X, axis=0)
    return X + 1.0 / n + S / (n * n) - r[:, None] / n - c[None, :] / n


def p2(X):
    return np.maximum(X, 0.0)


def p3(X):
    """Lemma (appendix, proof of Thm. 7): projection onto {Y1 = 0, Y^T 1 = 0}."""
    n = X.shape[0]
    S = np.sum(X)
    return X + S / (n * n) - np.sum(X, axis=1)[:, None] / n - np.sum(X, axis=0)[None, :] / n


# --------------------------------------------------------------------------
# Sec. 5.2: the dimension-invariant distance  gamma(X) = 1^T X 1 / n - 1.
# --------------------------------------------------------------------------
def gamma(Y):
    return float(np.sum(Y)) / Y.shape[0] - 1.0


@dataclass
class SDSNResult:
    D: np.ndarray
    sweeps: int
    gamma: float
    converged: bool
    gammas: list = field(default_factory=list)


# --------------------------------------------------------------------------
# Alg. 2 (SDSN).  Step 1: X^(0) = (theta/2) X / max(X).  Then repeat
# X <- P2(P1(X)) (eq. 8) and test gamma.
# Reading (iii): gamma is taken on the clamped result of each sweep (the
# appendix's lagged use of the previous sweep's sum is an optional saving),
# at least one sweep runs, and the loop stops at gamma <= gamma_tol or after
# max_sweeps sweeps.  Reading (iv): this is alternating projection; it is
# what FRAM computes, even where it differs from the exact P_D of eq. 4.
# --------------------------------------------------------------------------
def sdsn(X, theta, gamma_tol=1e-14, max_sweeps=200, keep_history=False):
    n = X.shape[0]
    m = float(np.max(X))
    if not m > 0:
        raise DegenerateError("max(X) <= 0 in SDSN step 1")
    Y = (theta / 2.0) * (X / m)
    g = math.inf
    hist = []
    k = 0
    while k < max_sweeps:
        Y = p2(p1(Y))
        k += 1
        g = gamma(Y)
        if keep_history:
            hist.append(g)
        if g <= gamma_tol:
            break
    return SDSNResult(Y, k, g, g <= gamma_tol, hist)


# --------------------------------------------------------------------------
# Eq. 4 / Thm. 1: the FRA solution itself, D_X^theta = argmin over D_n of
# ||D - (theta/2) X/max(X)||_F, which SDSN approximates (reading (iv)).  Not
# the paper's algorithm: an exact variant of step 6.
#
# With Y0 = (theta/2) X/max(X), the KKT conditions of this QP read
#   D = max(0, Y0 - a 1^T - 1 b^T),  D 1 = 1,  D^T 1 = 1
# for some multipliers a, b; any such D is the (unique) projection.  The
# multipliers come from block coordinate ascent on the concave dual: with b
# fixed, each a_i solves  sum_j max(0, Y0_ij - b_j - a_i) = 1, the threshold
# of a Euclidean projection onto the simplex (sort the row, find the
# largest k whose k-th value exceeds (sum of the first k - 1)/k); then each
# b_j likewise with a fixed.  `omega` > 1 over-relaxes both updates (falling
# back to 1 as soon as the residual grows); omega = 1 is the plain method.
# --------------------------------------------------------------------------
@dataclass
class FRAResult:
    D: np.ndarray
    sweeps: int
    residual: float      # max |row or column sum - 1| of D
    converged: bool
    a: np.ndarray
    b: np.ndarray


def simplex_thresholds(Z):
    """t_i with sum_j max(0, Z_ij - t_i) = 1 for every row i of Z."""
    Zs = -np.sort(-Z, axis=1)
    cs = np.cumsum(Zs, axis=1)
    k = np.arange(1, Z.shape[1] + 1)
    t = (cs - 1.0) / k
    active = Zs > t                     # true for k = 1 .. k*, false after
    kstar = active.sum(axis=1)          # >= 1: the largest value always qualifies
    return t[np.arange(Z.shape[0]), kstar - 1]


def fra_residual(D):
    return max(float(np.max(np.abs(D.sum(axis=1) - 1.0))),
               float(np.max(np.abs(D.sum(axis=0) - 1.0))))


def fra_exact(X, theta, tol=1e-12, max_sweeps=10000, omega=1.0):
    n = X.shape[0]
    m = float(np.max(X))
    if not m > 0:
        raise DegenerateError("max(X) <= 0 in the FRA scaling")
    Y0 = (theta / 2.0) * (X / m)
    a = np.zeros(n)
    b = np.zeros(n)
    res, prev, w = math.inf, math.inf, 1.0
    k = 0
    while k < max_sweeps:
        an = simplex_thresholds(Y0 - b[None, :])
        a = an if k == 0 else a + w * (an - a)
        bn = simplex_thresholds((Y0 - a[:, None]).T)
        b = bn if k == 0 else b + w * (bn - b)
        k += 1
        res = fra_residual(np.maximum(0.0, Y0 - a[:, None] - b[None, :]))
        if res <= tol:
            break
        w = omega if res < prev else 1.0
        prev = res
    D = np.maximum(0.0, Y0 - a[:, None] - b[None, :])
    return FRAResult(D, k, res, res <= tol, a, b)


# --------------------------------------------------------------------------
# Alg. 1 steps 7-8: damped update and the normalized Frobenius criterion
# (appendix, "Convergence Criterion of the Matching algorithm").
# --------------------------------------------------------------------------
def damped_update(N, D, alpha):
    N_new = (1.0 - alpha) * N + alpha * D
    delta = float(np.linalg.norm(N_new - N)) / float(np.linalg.norm(N_new))
    return N_new, delta


# --------------------------------------------------------------------------
# Eq. 2 / Alg. 1 step 10: M = argmin_P ||P - N||_F = argmax_P <P, N>.
# Kuhn's Hungarian method in its shortest-augmenting-path form with row and
# column potentials: rows are inserted one at a time and each insertion runs
# a Dijkstra search over reduced costs.  Reading (vi): ties are broken toward
# the lowest column index (first minimum of the scan).
# --------------------------------------------------------------------------
def lap_max(W):
    """Return perm (int64[n]) maximising sum_i W[i, perm[i]]."""
    W = np.asarray(W, dtype=np.float64)
    n = W.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    C = -W                                   # minimise cost
    INF = math.inf
    u = np.zeros(n + 1)                      # row potentials (1-based rows)
    v = np.zeros(n + 1)                      # column potentials, column 0 is a dummy
    p = np.zeros(n + 1, dtype=np.int64)      # p[j] = row matched to column j (0 = free)
    way = np.zeros(n + 1, dtype=np.int64)
    for i in range(1, n + 1):
        p[0] = i
        j0 = 0
        minv = np.full(n + 1, INF)
        used = np.zeros(n + 1, dtype=bool)
        while True:
            used[j0] = True
            i0 = p[j0]
            free = ~used[1:]
            cur = C[i0 - 1, :] - u[i0] - v[1:]
            better = free & (cur < minv[1:])
            minv[1:][better] = cur[better]
            way[1:][better] = j0
            cand = np.where(free, minv[1:], INF)
            j1 = int(np.argmin(cand)) + 1
            d = cand[j1 - 1]
            used_idx = np.flatnonzero(used)
            u[p[used_idx]] += d
            v[used_idx] -= d
            minv[1:][free] -= d
            j0 = j1
            if p[j0] == 0:
                break
        while j0 != 0:
            j1 = way[j0]
            p[j0] = p[j1]
            j0 = j1
    perm = np.empty(n, dtype=np.int64)
    for j in range(1, n + 1):
        perm[p[j] - 1] = j - 1
    return perm


# --------------------------------------------------------------------------
# Eq. 1 at a permutation: Phi(M) = 1/2 <M^T A M, A~> + lambda <M^T F, F~>,
# with M[i, perm[i]] = 1.  With K = F F~^T the node term is sum_i K[i, perm[i]].
# Evaluated as the O(n^2) gather 1/2 sum_ij A_ij A~_{perm(i) perm(j)}.
# --------------------------------------------------------------------------
def objective(A, B, perm, K=None, lam=1.0):
    perm = np.asarray(perm)
    val = 0.5 * float(np.sum(A * B[np.ix_(perm, perm)]))
    if K is not None:
        val += lam * float(np.sum(K[np.arange(len(perm)), perm]))
    return val


# Sec. 7 "Criteria": matching error 1/2 ||A - M A~ M^T||_F (edge term only),
# with (M A~ M^T)_ij = A~_{perm(i) perm(j)}.
def matching_error(A, B, perm):
    perm = np.asarray(perm)
    return 0.5 * float(np.linalg.norm(A - B[np.ix_(perm, perm)]))


# Sec. 7 "Criteria": accuracy n_c / n over nodes that have a true partner.
def accuracy(perm, truth):
    truth = np.asarray(truth)
    valid = truth >= 0
    if not np.any(valid):
        return 1.0
    return float(np.mean(np.asarray(perm)[valid] == truth[valid]))


@dataclass
class FramResult:
    N: np.ndarray
    perm: np.ndarray
    outer_iters: int
    total_sweeps: int
    delta: float
    gamma: float
    sdsn_converged_last: bool
    objective: float
    match_error: float
    sweeps: list = field(default_factory=list)
    deltas: list = field(default_factory=list)


# --------------------------------------------------------------------------
# Alg. 1 (FRAM) end to end.
#   steps 2-3 prescale; step 1 initial N (reading (i));
#   loop (step 4) while delta > delta_tol, at most max_outer times
#   (reading (ii): delta^(0) is undefined, so the first iteration always runs):
#     step 5  X = A N A~ + lambda K
#     step 6  D = SDSN(X, theta)
#     step 7  N = (1 - alpha) N + alpha D
#     step 8  delta = ||N_t - N_{t-1}||_F / ||N_t||_F
#   step 10 discretise N with the Hungarian method (eq. 2);
#   objective and matching error on the unscaled inputs.
# --------------------------------------------------------------------------
def fram(A, B, K=None, lam=1.0, alpha=0.95, theta=10.0, delta_tol=1e-6, max_outer=100,
         gamma_tol=1e-14, max_sweeps=200, validate_inputs=True, projection="sdsn",
         exact_tol=None, omega=1.0):
    """projection="sdsn" is Alg. 1 as printed; "exact" replaces step 6 by the
    exact FRA solution (fra_exact, stopped at exact_tol, default
    max(gamma_tol, 8 n eps), after at most max_sweeps sweeps); its residual
    stands in for gamma in the result."""
    A0 = np.asarray(A, dtype=np.float64)
    B0 = np.asarray(B, dtype=np.float64)
    K0 = None if K is None else np.asarray(K, dtype=np.float64)
    if validate_inputs:
        validate(A0, B0, K0)
    n = A0.shape[0]
    As, Bs, Ks, _ = prescale(A0, B0, K0)
    N = initial_assignment(n, K0 is not None)
    total = 0
    delta = math.inf
    g = math.nan
    conv = False
    sweeps, deltas = [], []
    t = 0
    while t < max_outer:
        X = gradient(As, N, Bs, Ks, lam)
        if projection == "exact":
            tol = exact_tol if exact_tol is not None else max(gamma_tol, 8 * n * 2.0 ** -52)
            res = fra_exact(X, theta, tol, max_sweeps, omega)
            g = res.residual
        else:
            res = sdsn(X, theta, gamma_tol, max_sweeps)
            g = res.gamma
        N, delta = damped_update(N, res.D, alpha)
        t += 1
        total += res.sweeps
        conv = res.converged
        sweeps.append(res.sweeps)
        deltas.append(delta)
        if delta <= delta_tol:
            break
    perm = lap_max(N)
    return FramResult(N, perm, t, total, delta, g, conv,
                      objective(A0, B0, perm, K0, lam), matching_error(A0, B0, perm),
                      sweeps, deltas)
