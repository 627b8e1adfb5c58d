"""Pins for the oracle's codebook training (§2.3.1 Multi-D-ADC, §3.2 HBPQ local
codebooks) on learn sets whose codebooks can be written down by hand.

The construction: when K equals the number of training vectors and those vectors
are distinct, Lloyd's K-means started from them keeps every vector as its own
centroid, so the residual codebook R_k must equal, row for row, the learn set's
displacements in sub-space k.  Which displacements those are is what the tests
pin: x - [c^1_i; c^2_j] with the coarse centroids of the point's own cell.  The
expected values are written out from the construction (means of index sets,
formulas in the loop variables), never by calling the oracle's quantizers.
"""
import numpy as np

from oracle import bpq_oracle as O


def grid_learn():
    """256 learn points of D = 4: first half (a, b), second half (2a + 100, b + 50),
    a, b = 0..15 in row-major order.  Every half and every 2-D sub-vector is
    distinct across the 256 points."""
    a, b = np.divmod(np.arange(256), 16)
    return np.stack([a, b, 2 * a + 100, b + 50], axis=1), a, b


def test_single_cell_codebooks_by_hand():
    """T = 1: C^1 and C^2 are the rounded-half-up means of the halves, and with
    M = 2 (one sub-quantizer per half) R_0, R_1 are the displacements from them.
      mean of a and b over the grid = 7.5 -> 8 (half up);
      second half mean = (2 * 7.5 + 100, 7.5 + 50) = (115, 57.5) -> (115, 58)."""
    learn, a, b = grid_learn()
    cb = O.train_multi_d_adc(learn, T=1, M=2, iters=3)
    assert cb.C1.tolist() == [[8, 8]]
    assert cb.C2.tolist() == [[115, 58]]
    assert cb.R.shape == (2, 256, 2)
    assert cb.R[0].tolist() == np.stack([a - 8, b - 8], 1).tolist()
    assert cb.R[1].tolist() == np.stack([2 * a - 15, b - 8], 1).tolist()


def test_single_cell_codebooks_reject_plausible_mistakes():
    """The expected codebooks of the T = 1 case differ from what a raw-sub-vector
    residual training (R_k on x instead of x - c), a second half quantized against
    C^1, or a floor-rounded mean would give."""
    learn, a, b = grid_learn()
    cb = O.train_multi_d_adc(learn, T=1, M=2, iters=3)
    raw = np.stack([a, b], 1)
    assert cb.R[0].tolist() != raw.tolist()
    wrong_half = np.stack([2 * a + 100 - 8, b + 50 - 8], 1)
    assert cb.R[1].tolist() != wrong_half.tolist()
    assert cb.C1.tolist() != [[7, 7]]


def two_cell_learn():
    """256 learn points of D = 4 in two well-separated groups per half.
    Point n = 16 a + b (a, b = 0..15):
      first half  (40 g + a, b)              g = b % 2
      second half (100 + 50 h + b, a)        h = (a + b) % 2
    Every half is distinct across the points.  Points 0 and 1 (the K-means starts)
    lie in different groups in both halves, and the groups are far enough apart
    that the first assignment already separates them."""
    a, b = np.divmod(np.arange(256), 16)
    g, h = b % 2, (a + b) % 2
    x = np.stack([40 * g + a, b, 100 + 50 * h + b, a], axis=1)
    return x, a, b, g, h


def half_up(v):
    """Rounded-half-up integer mean of a list of ints."""
    s, n = int(sum(int(t) for t in v)), len(v)
    return (2 * s + n) // (2 * n)


def test_two_cell_coarse_centroids_and_displacements():
    """T = 2: the coarse centroids are the rounded means of the two groups of each
    half, and R_k holds, row for row, x - [c^1_i; c^2_j] with the centroids of the
    point's own cell (duplicate displacements tie to the lower index and the higher
    copy keeps its start, so the rows survive Lloyd unchanged)."""
    x, a, b, g, h = two_cell_learn()
    cb = O.train_multi_d_adc(x, T=2, M=2, iters=6)
    mean1 = {gg: [half_up(x[g == gg, d]) for d in (0, 1)] for gg in (0, 1)}
    mean2 = {hh: [half_up(x[h == hh, d]) for d in (2, 3)] for hh in (0, 1)}
    assert mean1 == {0: [8, 7], 1: [48, 8]} and mean2 == {0: [108, 8], 1: [158, 8]}
    assert cb.C1.tolist() == [mean1[0], mean1[1]]  # starts: point 0 (g = 0), point 1 (g = 1)
    assert cb.C2.tolist() == [mean2[0], mean2[1]]
    c1 = np.array([mean1[v] for v in g])
    c2 = np.array([mean2[v] for v in h])
    assert cb.R[0].tolist() == (x[:, :2] - c1).tolist()
    assert cb.R[1].tolist() == (x[:, 2:] - c2).tolist()
    # a displacement from the global mean, or from the other group's centroid,
    # would not match
    assert cb.R[0].tolist() != (x[:, :2] - np.array([half_up(x[:, 0]), half_up(x[:, 1])])).tolist()
    assert cb.R[1].tolist() != (x[:, 2:] - np.array([mean2[1 - v] for v in h])).tolist()


def test_local_codebooks_by_hand():
    """HBPQ local training (Eqs. 10-11): the codebooks of a half-cell are learned
    only on the displacements of the learn points that fall in it, starting from
    the global codebook.
      * Half-cell 0 of each half holds the 256 grid points, whose displacements are
        exactly the global codebook: a fixed point, so Q^0_0 = R_0 and S^0_0 = R_1.
      * Half-cell 1 of the first half holds two points with displacements (20, 20)
        and (21, 20); both are nearest to codeword 255 = (7, 7), which moves to their
        rounded mean (21, 20); every other codeword keeps its start.
      * Half-cell 1 of the second half holds (30, -30) and (31, -30); both are
        nearest to codeword 240 = (15, -8), which moves to (31, -30).
    Training a half-cell on every learn point, or on raw sub-vectors, moves other
    codewords and fails these equalities."""
    learn, a, b = grid_learn()
    glob = O.train_multi_d_adc(learn, T=1, M=2, iters=2)
    C1 = np.array([[8, 8], [200, 200]])
    C2 = np.array([[115, 58], [10, 250]])
    cb = O.Codebooks(D=4, T=2, M=2, C1=C1, C2=C2, R=glob.R)
    extra = np.array([[220, 220, 40, 220], [221, 220, 41, 220]])
    loc = O.train_hbpq_local(np.concatenate([learn, extra]), cb, iters=3)
    assert loc.Q.shape == (2, 1, 256, 2) and loc.S.shape == (2, 1, 256, 2)
    R0 = np.stack([a - 8, b - 8], 1)
    R1 = np.stack([2 * a - 15, b - 8], 1)
    assert np.array_equal(glob.R[0], R0) and np.array_equal(glob.R[1], R1)
    assert np.array_equal(loc.Q[0, 0], R0) and np.array_equal(loc.S[0, 0], R1)
    want_q1 = R0.copy()
    want_q1[255] = [21, 20]
    want_s1 = R1.copy()
    want_s1[240] = [31, -30]
    assert np.array_equal(loc.Q[1, 0], want_q1)
    assert np.array_equal(loc.S[1, 0], want_s1)
