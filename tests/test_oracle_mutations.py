"""Planted mistakes in the oracle (on the CPU): each mutant must fail the pin
that is meant to catch it, so a plausible slip in the oracle cannot pass
unnoticed.  The mutants live only inside these tests."""
import numpy as np
import pytest

import oracle as o
from test_oracle_pins import brute_lap, kkt_affine_projection, rand_mat


def _p1_kkt_ok(p1):
    for n in (3, 5):
        X = rand_mat(n, 2) * 3 - 1
        if np.max(np.abs(p1(X) - kkt_affine_projection(X))) > 1e-13:
            return False
    return True


def _p1_swapped(X):          # transposed operand: row and column sums exchanged
    n = X.shape[0]
    return X + 1 / n + X.sum() / n**2 - X.sum(0)[:, None] / n - X.sum(1)[None, :] / n


def _p1_dropped(X):          # dropped term: S/n^2 missing
    n = X.shape[0]
    return X + 1 / n - X.sum(1)[:, None] / n - X.sum(0)[None, :] / n


def _p1_sign(X):             # wrong sign on the column term
    n = X.shape[0]
    return X + 1 / n + X.sum() / n**2 - X.sum(1)[:, None] / n + X.sum(0)[None, :] / n


def test_reference_p1_passes():
    assert _p1_kkt_ok(o.p1)


@pytest.mark.parametrize("mutant", [_p1_swapped, _p1_dropped, _p1_sign])
def test_p1_mutants_fail_kkt_pin(mutant):
    assert not _p1_kkt_ok(mutant)


def _grad_fd_ok(grad):
    n = 5
    A = rand_mat(n, 1, asym=False)
    B = rand_mat(n, 2, asym=False)
    N = rand_mat(n, 3)
    phi = lambda M: 0.5 * np.sum((M.T @ A @ M) * B)
    G = grad(A, N, B)
    h = 1e-6
    for i, j in [(0, 1), (2, 4), (3, 0)]:
        E = np.zeros((n, n))
        E[i, j] = h
        if abs((phi(N + E) - phi(N - E)) / (2 * h) - G[i, j]) > 1e-7:
            return False
    return True


def test_gradient_mutant_fails_fd_pin():
    assert _grad_fd_ok(lambda A, N, B: o.gradient(A, N, B))
    assert not _grad_fd_ok(lambda A, N, B: A @ N.T @ B)


def test_lap_mutant_fails_brute_force_pin():
    W = rand_mat(6, 8)
    _, best = brute_lap(W)
    good = o.lap_max(W)
    bad = o.lap_max(-W)                  # minimises instead of maximising
    assert abs(W[np.arange(6), good].sum() - best) < 1e-12
    assert abs(W[np.arange(6), bad].sum() - best) > 1e-6


def test_sdsn_lagged_gamma_mutant_fails_golden():
    # Literal reading of Alg. 2 (test gamma of the matrix *before* the sweep,
    # including the unclamped scaled input) stops one sweep late on the
    # hand-derived example; the golden sweep count catches it.
    X = np.eye(2)
    Y = 5.0 * X
    k, g = 0, np.inf
    while g > 1e-14 and k < 200:
        g = Y.sum() / 2 - 1            # lagged: measured before this sweep
        Y = o.p2(o.p1(Y))
        k += 1
    assert k != o.sdsn(X, 10.0, 1e-14, 200).sweeps


def _thresholds_ok(thr):
    rng = np.random.default_rng(3)
    Z = rng.normal(size=(12, 9))
    t = thr(Z)
    return np.max(np.abs(np.maximum(0.0, Z - t[:, None]).sum(1) - 1.0)) <= 1e-12


def _thr_off_by_one(Z):      # k* - 1 used as the count of the active set
    Zs = -np.sort(-Z, axis=1)
    cs = np.cumsum(Zs, axis=1)
    k = np.arange(1, Z.shape[1] + 1)
    t = (cs - 1.0) / k
    kstar = np.maximum((Zs > t).sum(axis=1) - 1, 1)
    return t[np.arange(Z.shape[0]), kstar - 1]


def _thr_no_sort(Z):         # prefix sums of the unsorted row
    cs = np.cumsum(Z, axis=1)
    k = np.arange(1, Z.shape[1] + 1)
    t = (cs - 1.0) / k
    kstar = (Z > t).sum(axis=1)
    return t[np.arange(Z.shape[0]), kstar - 1]


def test_reference_thresholds_pass():
    assert _thresholds_ok(o.simplex_thresholds)


@pytest.mark.parametrize("mutant", [_thr_off_by_one, _thr_no_sort])
def test_threshold_mutants_fail_their_pin(mutant):
    assert not _thresholds_ok(mutant)
