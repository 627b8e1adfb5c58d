"""Pins for the oracle's OPQ variant (the "optimized" OMulti-D-OADC of §2.3 used in
the paper's experiments; parametric OPQ learner)."""
import numpy as np
import pytest

from oracle import bpq_oracle as O


def test_eigenvalue_allocation_by_hand():
    """Dealt in descending order to the subspace with the smallest sum of logs:
    8 -> 0; 4 -> 1 (log 4 < log 8); 2 -> 1 (log 4 < log 8); 1 -> 0 (the only one left)."""
    assert O.allocate_eigenvalues([8, 4, 2, 1], 2) == [[0, 3], [1, 2]]
    assert O.allocate_eigenvalues([1, 2, 4, 8], 2) == [[3, 0], [2, 1]]
    # ties: equal sums go to the lower subspace while it has room
    assert O.allocate_eigenvalues([1, 1, 1, 1], 2) == [[0, 1], [2, 3]]
    # four subspaces of one dimension: one eigenvalue each, largest first
    assert O.allocate_eigenvalues([3, 9, 1, 5], 4) == [[1], [3], [0], [2]]


def planted(scales=(4, 3, 2, 1)):
    """Z: every sign pattern of the scales (mean 0, covariance exactly
    diag(scales^2)); X = Z Q^T with Q two 45-degree plane rotations."""
    d = len(scales)
    signs = np.array([[1 if (m >> b) & 1 else -1 for b in range(d)] for m in range(2 ** d)])
    Z = signs * np.array(scales, dtype=np.float64)
    c = np.sqrt(0.5)
    Q = np.array([[c, -c, 0, 0], [c, c, 0, 0], [0, 0, c, -c], [0, 0, c, c]])
    return Z, Q, Z @ Q.T


def test_opq_rotation_recovers_planted_rotation():
    """Eigenvalues 16, 9, 4, 1 are dealt as [16, 1 | 9, 4]: the rows of the rotation are
    the columns of Q for 16, 1, 9, 4 (signs fixed by the largest component), so the
    rotated data are the planted coordinates in that order, up to sign."""
    Z, Q, X = planted()
    R = O.opq_rotation(X, 2)
    assert np.allclose(R @ R.T, np.eye(4), atol=1e-12)
    Y = X @ R.T
    for row, col in zip(range(4), (0, 3, 1, 2)):
        assert np.allclose(np.abs(Y[:, row]), np.abs(Z[:, col]), atol=1e-9)
    # each row's largest-magnitude component is positive
    for v in R:
        assert v[np.argmax(np.abs(v))] > 0


def test_opq_rotation_diagonalizes_random_covariance():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(8, 8))
    X = rng.normal(size=(5000, 8)) @ A
    R = O.opq_rotation(X, 4)
    assert np.allclose(R @ R.T, np.eye(8), atol=1e-10)
    Xc = X - X.mean(0)
    C = R @ (Xc.T @ Xc / len(X)) @ R.T
    off = C - np.diag(np.diag(C))
    assert np.abs(off).max() < 1e-8 * np.abs(C).max()


def small_learn(seed=4, n=3000, D=8):
    """Correlated integer data from one fixed distribution (independent coordinates of
    unequal spread, then one fixed rotation); `seed` draws the sample."""
    Qm, _ = np.linalg.qr(np.random.default_rng(99).normal(size=(D, D)))
    Z = np.random.default_rng(seed).normal(size=(n, D)) * np.array([60, 40, 25, 15, 10, 6, 4, 2])[:D]
    return np.floor(Z @ Qm.T + 128.5).astype(np.int64)


def test_identity_rotations_reduce_to_multi_d_adc():
    learn = small_learn()
    cb = O.train_multi_d_adc(learn, T=4, M=4, iters=3)
    I8, I4 = np.eye(8), np.eye(4)
    cbi = O.train_opq(learn, T=4, M=4, iters=3, rotations=(I8, I4, I4))
    for n in ("C1", "C2", "R"):
        assert np.array_equal(getattr(cb, n), getattr(cbi, n))
    X = small_learn(seed=5, n=500)
    a, b = O.encode_multi_d_adc(X, cb), O.encode_multi_d_adc(X, cbi)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    q = X[:3].astype(np.float64) + 0.25
    ia = O.build_index(cb, X)
    ib = O.build_index(cbi, X)
    for qq in q:
        ra = O.search_one(ia, qq, 200, 10, "fbpq")
        rb = O.search_one(ib, qq, 200, 10, "fbpq")
        assert np.array_equal(ra[0], rb[0]) and np.allclose(ra[1], rb[1], rtol=1e-12)


@pytest.fixture(scope="module")
def opq_index():
    learn = small_learn()
    cb = O.train_opq(learn, T=4, M=4, iters=3)
    X = small_learn(seed=6, n=2000)
    return cb, O.build_index(cb, X), X


def test_opq_fbpq_equals_reconstruction(opq_index):
    """Eq. 8 + Eq. 9 with the rotated query and centroids equals the distance to the
    reconstruction rot0^T(c + [rot1^T r^1; rot2^T r^2]) in the original space."""
    cb, idx, X = opq_index
    assert cb.rotated and np.allclose(cb.rot0 @ cb.rot0.T, np.eye(8), atol=1e-10)
    lists = idx.lists
    pos = np.arange(0, len(lists.ids), 3)
    cell_of = np.searchsorted(lists.offsets, pos, side="right") - 1
    for q in X[:5].astype(np.float64) + 0.3:
        a = O.dist_fbpq(q, cb, idx.tables, cell_of, lists.codes[pos])
        b = O.dist_reconstruct(q, O.reconstruct(cb, cell_of, lists.codes[pos]))
        assert np.allclose(a, b, rtol=1e-9, atol=1e-7)
    ra = O.search(idx, X[:8], 400, 10, "fbpq")
    rb = O.search(idx, X[:8], 400, 10, "recon")
    assert np.array_equal(ra[0], rb[0]) and np.allclose(ra[1], rb[1], rtol=1e-9)


def test_opq_dropped_rotation_is_detected(opq_index):
    """The residual tables with the unrotated query (a plausible mistake) differ."""
    cb, idx, X = opq_index
    lists = idx.lists
    pos = np.arange(0, len(lists.ids), 7)
    cell_of = np.searchsorted(lists.offsets, pos, side="right") - 1
    wrong = O.Codebooks(D=cb.D, T=cb.T, M=cb.M, C1=cb.C1, C2=cb.C2, R=cb.R, rot0=cb.rot0,
                        rot1=np.eye(4), rot2=np.eye(4))
    q = X[0].astype(np.float64)
    a = O.dist_fbpq(q, wrong, O.fbpq_tables(wrong), cell_of, lists.codes[pos])
    b = O.dist_reconstruct(q, O.reconstruct(cb, cell_of, lists.codes[pos]))
    assert not np.allclose(a, b, rtol=1e-6)


def test_opq_lowers_encoding_error_on_correlated_data():
    """On rotated data with unequal variances, OPQ encodes better than axis-aligned PQ."""
    learn = small_learn(n=6000)
    X = small_learn(seed=8, n=3000)
    plain = O.train_multi_d_adc(learn, T=4, M=4, iters=5)
    opq = O.train_opq(learn, T=4, M=4, iters=5)
    assert O.encoding_error(opq, X).mean() < 0.9 * O.encoding_error(plain, X).mean()
