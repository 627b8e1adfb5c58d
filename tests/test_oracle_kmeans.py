"""Pins for the oracle's k-means and quantizers (§2.1, §2.3.1) against hand
computations and brute force."""
import itertools

import numpy as np
import pytest

from oracle import bpq_oracle as O


def test_sq_dists_equals_plain_sum_of_squares():
    rng = np.random.default_rng(0)
    X = rng.integers(-255, 256, size=(50, 16))
    C = rng.integers(-255, 256, size=(30, 16))
    plain = np.array([[sum((int(a) - int(b)) ** 2 for a, b in zip(x, c)) for c in C] for x in X])
    assert np.array_equal(O.sq_dists(X, C), plain.astype(np.float64))


def test_nearest_brute_force_with_ties():
    C = np.array([[0, 0], [2, 0], [0, 2], [2, 0]])
    X = np.array([[1, 0], [1, 1], [3, 0], [0, 1], [5, 5]])
    # [1,0] ties codewords 0 and 1 -> 0; [1,1] ties 0,1,2 -> 0; [3,0] ties 1 and 3 -> 1
    assert list(O.nearest(X, C)) == [0, 0, 1, 0, 1]
    rng = np.random.default_rng(1)
    X = rng.integers(0, 8, size=(200, 3))
    C = rng.integers(0, 8, size=(17, 3))
    for x, a in zip(X, O.nearest(X, C)):
        d = [sum((int(p) - int(q)) ** 2 for p, q in zip(x, c)) for c in C]
        assert a == d.index(min(d))


def test_rounded_mean_half_up_and_negative():
    sums = np.array([[3], [5], [-3], [-5], [7], [-1]])
    counts = np.array([2, 2, 2, 2, 3, 2])
    # 1.5 -> 2, 2.5 -> 3, -1.5 -> -1, -2.5 -> -2, 7/3 -> 2, -0.5 -> 0
    assert rounded_list(O.rounded_mean(sums, counts)) == [2, 3, -1, -2, 2, 0]


def rounded_list(a):
    return [int(v) for v in np.asarray(a).ravel()]


def test_kmeans_two_separated_clusters_1d():
    X = np.array([[0], [2], [4], [100], [104], [107]])
    C, hist = O.kmeans(X, 2, 5, init=np.array([[0], [4]]))
    # first step: {0,2} -> 1, {4,100,104,107} -> 78.75 -> 79; then clusters separate
    assert sorted(rounded_list(C)) == [2, 104]  # (0+2+4)/3 = 2, (100+104+107)/3 = 103.67 -> 104
    assert all(a >= b for a, b in zip(hist, hist[1:]))


def test_kmeans_2d_exact_means_and_empty_cluster():
    X = np.array([[0, 0], [0, 2], [2, 0], [2, 2], [10, 10], [10, 12], [12, 10], [12, 12]])
    init = np.array([[0, 0], [10, 10], [50, 50]])
    C, _ = O.kmeans(X, 3, 4, init=init)
    assert C.tolist() == [[1, 1], [11, 11], [50, 50]]  # empty third cluster keeps its centroid


def test_kmeans_default_init_first_rows():
    X = np.array([[5], [1], [9], [5]])
    C, _ = O.kmeans(X, 2, 0)
    assert C.tolist() == [[5], [1]]
    with pytest.raises(ValueError):
        O.kmeans(X[:1], 2, 1)


def test_kmeans_fixed_point_and_monotone_on_random_data():
    rng = np.random.default_rng(3)
    X = rng.integers(0, 256, size=(500, 4))
    C, hist = O.kmeans(X, 8, 25)
    assert all(a >= b for a, b in zip(hist, hist[1:]))
    # at convergence every centroid is the rounded mean of its own cluster
    a = O.nearest(X, C)
    for c in range(8):
        if (a == c).any():
            m = X[a == c].sum(0)
            n = (a == c).sum()
            assert C[c].tolist() == [(2 * int(v) + int(n)) // (2 * int(n)) for v in m]


def test_rounded_mean_is_best_integer_centroid():
    """The rounded mean minimises sum ||x - c||^2 over integer c (separable per
    coordinate), which is what keeps integer-grid Lloyd monotone."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        X = rng.integers(-20, 20, size=(7, 2))
        c = O.rounded_mean(X.sum(0)[None, :], np.array([len(X)]))[0]
        best = min(itertools.product(range(-25, 26), repeat=2),
                   key=lambda p: ((X - np.array(p)) ** 2).sum())
        assert ((X - c) ** 2).sum() == ((X - np.array(best)) ** 2).sum()
