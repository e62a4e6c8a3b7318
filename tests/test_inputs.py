"""The seeded input generators do what their recipe states (CPU only).

Every workload the tests and the bench use comes from ``fram_inputs``; these
checks pin the stated structure: symmetric, nonnegative, zero-diagonal FP64
graphs; the planted relabelling B[p_i, p_j] = A[i, j]; the edge counts the
flips preserve; the social graph's scale and degree tail; the Gaussian
kernel's median-distance sigma; the keypoint padding; the serving stream's
size law.  No method arithmetic is involved."""
import numpy as np
import pytest

import fram_inputs as fi


def assert_graph(M, n):
    assert M.dtype == np.float64 and M.shape == (n, n) and M.flags.c_contiguous
    assert np.array_equal(M, M.T)
    assert np.all(M >= 0) and np.all(np.isfinite(M))
    assert np.all(np.diag(M) == 0)


def upper_edges(M):
    return int(np.count_nonzero(np.triu(M, 1)))


@pytest.mark.parametrize("make", [
    lambda: fi.er_pair(60, 0.2, noise=0.05, flip_frac=0.05, seed=1),
    lambda: fi.small_er_pair(3),
    lambda: fi.social_pair(300, 2000, 0.05, seed=2),
    lambda: fi.gaussian_pair(80, seed=4),
    lambda: fi.attributed_pair(70, d=16, seed=5),
    lambda: fi.keypoint_pair(np.random.default_rng(6)),
    lambda: fi.serving_pair(90, seed=7),
])
def test_every_generator_gives_valid_graphs(make):
    g = make()
    n = g.n
    assert_graph(g.A, n)
    assert_graph(g.B, n)
    assert g.truth.dtype == np.int64 and g.truth.shape == (n,)
    real = g.truth[g.truth >= 0]
    assert np.unique(real).size == real.size and np.all(real < n)


def test_noiseless_er_pair_is_the_planted_relabelling():
    g = fi.er_pair(40, 0.3, seed=11)
    p = g.truth
    assert np.array_equal(g.B[np.ix_(p, p)], g.A)          # B[p_i, p_j] = A[i, j]
    assert sorted(p.tolist()) == list(range(40))


def test_er_edge_noise_touches_existing_edges_only():
    g = fi.er_pair(50, 0.2, noise=0.05, seed=12)
    p = g.truth
    Bp = g.B[np.ix_(p, p)]                                   # back in A's labels
    assert np.all(Bp[g.A == 0] == 0)                         # no new edges
    assert np.any(Bp != g.A)                                 # weights moved


def test_er_flips_preserve_the_edge_count():
    g0 = fi.er_pair(120, 0.1, seed=13)
    g = fi.er_pair(120, 0.1, flip_frac=0.1, seed=13)
    assert upper_edges(g.B) == upper_edges(g0.A)
    p = g.truth
    Bp = g.B[np.ix_(p, p)]
    moved = np.count_nonzero(np.triu((Bp > 0) != (g.A > 0), 1))
    k = int(round(0.1 * upper_edges(g0.A)))
    assert moved == 2 * k                                    # k deleted, k added


def test_social_pair_scale_and_heavy_tail():
    n, m = 1500, 20000
    g = fi.social_pair(n, m, 0.0, seed=14)
    e = upper_edges(g.A)
    assert set(np.unique(g.A)) <= {0.0, 1.0}                  # unweighted
    assert abs(e - m) <= 5 * np.sqrt(m)                      # expected edge count m
    assert g.meta["edges"] == e
    deg = g.A.sum(1)
    assert deg.max() >= 8 * np.median(deg)                   # power-law tail
    p = g.truth
    assert np.array_equal(g.B[np.ix_(p, p)], g.A)            # no flips: exact relabelling


def test_social_pair_flips_preserve_the_edge_count():
    g = fi.social_pair(400, 3000, 0.05, seed=15)
    assert upper_edges(g.B) == upper_edges(g.A)


def test_gaussian_kernel_uses_the_median_distance():
    # A = exp(-d^2 / sigma^2) with sigma the median pairwise distance, so the
    # median off-diagonal entry is exp(-1) (an odd number of pairs: n = 51).
    g = fi.gaussian_pair(51, seed=16)
    iu = np.triu_indices(51, 1)
    assert iu[0].size % 2 == 1
    assert abs(np.median(g.A[iu]) - np.exp(-1.0)) < 1e-12
    assert np.all(g.A[iu] > 0) and np.all(g.A[iu] <= 1)


def test_attributed_descriptors_are_unit_nonnegative_and_planted():
    g = fi.attributed_pair(60, d=32, desc_noise=0.0, seed=17)
    for F in (g.F, g.Ft):
        assert np.all(F >= 0)
        assert np.allclose(np.linalg.norm(F, axis=1), 1.0, atol=1e-12)
    assert np.allclose(g.Ft[g.truth], g.F, atol=1e-12)       # no noise: same descriptor


def test_keypoint_padding_and_truth():
    rng = np.random.default_rng(18)
    for _ in range(50):
        g = fi.keypoint_pair(rng)
        n, m = g.n, g.meta["inliers"]
        assert 10 <= n <= 64
        assert np.all(g.truth[:m] >= 0) and np.all(g.truth[m:] == -1)
        # dummy nodes are isolated
        o1 = g.meta["o1"]
        assert np.all(g.A[m + o1:] == 0)
        real2 = np.count_nonzero(g.B.sum(1) > 0)
        assert real2 <= m + g.meta["o2"]


def test_serving_stream_size_law_and_arrivals():
    t, specs = fi.serving_stream(4000, seed=19, rate=5.0)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 4000 - 1 / 5.0) < 0.02                # mean gap 1/rate
    ns = np.array([s[0] for s in specs])
    assert ns.min() >= 20 and ns.max() <= 2048
    ln = np.log(ns)                                          # log-uniform on [20, 2048]
    assert abs(np.median(ln) - 0.5 * (np.log(20) + np.log(2048))) < 0.15
