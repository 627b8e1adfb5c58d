"""Pins for encoding and the inverted multi-index layout (§2.3.2, §3.2)."""
import numpy as np

from oracle import bpq_oracle as O


def small_codebooks(rng, D=8, T=4, M=4, local=False):
    h, s = D // 2, D // M
    cb = O.Codebooks(D=D, T=T, M=M,
                     C1=rng.integers(0, 256, size=(T, h)), C2=rng.integers(0, 256, size=(T, h)),
                     R=rng.integers(-60, 61, size=(M, O.KSUB, s)))
    if local:
        cb.Q = rng.integers(-60, 61, size=(T, M // 2, O.KSUB, s))
        cb.S = rng.integers(-60, 61, size=(T, M // 2, O.KSUB, s))
    return cb


def brute_encode(x, cb, local=False):
    """Cell and codes by trying every codeword, with Python ints."""
    h, s, m2 = cb.D // 2, cb.sub, cb.M // 2
    x = [int(v) for v in x]

    def arg(vec, book):
        d = [sum((a - int(b)) ** 2 for a, b in zip(vec, w)) for w in book]
        return d.index(min(d))

    i, j = arg(x[:h], cb.C1), arg(x[h:], cb.C2)
    disp = [a - int(b) for a, b in zip(x, list(cb.C1[i]) + list(cb.C2[j]))]
    codes = []
    for k in range(cb.M):
        book = (cb.Q[i, k] if k < m2 else cb.S[j, k - m2]) if local else cb.R[k]
        codes.append(arg(disp[k * s:(k + 1) * s], book))
    return i * cb.T + j, codes


def test_encode_multi_d_adc_brute_force():
    rng = np.random.default_rng(10)
    cb = small_codebooks(rng)
    X = rng.integers(0, 256, size=(40, 8))
    cells, codes = O.encode_multi_d_adc(X, cb)
    for n in range(len(X)):
        c, k = brute_encode(X[n], cb)
        assert cells[n] == c and codes[n].tolist() == k


def test_encode_hbpq_brute_force():
    rng = np.random.default_rng(11)
    cb = small_codebooks(rng, local=True)
    X = rng.integers(0, 256, size=(40, 8))
    cells, codes = O.encode_hbpq(X, cb)
    for n in range(len(X)):
        c, k = brute_encode(X[n], cb, local=True)
        assert cells[n] == c and codes[n].tolist() == k


def test_build_lists_layout():
    cells = np.array([5, 1, 5, 0, 1, 5])
    ids = np.array([10, 11, 12, 13, 14, 15])
    codes = np.arange(6, dtype=np.uint8)[:, None].repeat(2, 1)
    L = O.build_lists(cells, codes, ids, T=3)
    assert L.offsets.tolist() == [0, 1, 3, 3, 3, 3, 6, 6, 6, 6]
    assert L.ids.tolist() == [13, 11, 14, 10, 12, 15]
    assert L.codes[:, 0].tolist() == [3, 1, 4, 0, 2, 5]
    assert L.counts().sum() == 6


def literal_codebooks():
    """D = 4, T = 2, M = 2 codebooks with entries chosen by hand:
    C^1 = [[1, 2], [3, 4]], C^2 = [[5, 6], [7, 8]], R_0[t] = (t, -t), R_1[t] = (2t, 1);
    local codebooks Q^i_0[t] = (10 i + t, 0), S^j_0[t] = (0, -t - j)."""
    t = np.arange(O.KSUB)
    R = np.stack([np.stack([t, -t], 1), np.stack([2 * t, np.ones_like(t)], 1)])
    Q = np.stack([np.stack([10 * i + t, 0 * t], 1)[None] for i in range(2)])
    S = np.stack([np.stack([0 * t, -t - j], 1)[None] for j in range(2)])
    return O.Codebooks(D=4, T=2, M=2, C1=np.array([[1, 2], [3, 4]]), C2=np.array([[5, 6], [7, 8]]), R=R, Q=Q, S=S)


def test_reconstruct_literal_equation_7():
    """Eq. 7 by hand: cell (i, j) = (1, 0), code (3, 5):
    [c^1_1; c^2_0] + [R_0[3]; R_1[5]] = [3, 4, 5, 6] + [3, -3, 10, 1] = [6, 1, 15, 7]."""
    cb = literal_codebooks()
    xh = O.reconstruct(cb, np.array([1 * 2 + 0]), np.array([[3, 5]]))
    assert xh.tolist() == [[6.0, 1.0, 15.0, 7.0]]


def test_reconstruct_hbpq_literal():
    """HBPQ reconstruction (§3.2) by hand: cell (1, 1), code (3, 5) uses Q^1_0 and
    S^1_0: [3, 4] + (13, 0) and [7, 8] + (0, -6) -> [16, 4, 7, 2]."""
    cb = literal_codebooks()
    xh = O.reconstruct_hbpq(cb, np.array([1 * 2 + 1]), np.array([[3, 5]]))
    assert xh.tolist() == [[16.0, 4.0, 7.0, 2.0]]


def test_train_shapes_and_local_training_improves_distortion():
    rng = np.random.default_rng(13)
    learn = rng.integers(0, 256, size=(3000, 8)) // np.array([1, 1, 4, 4, 1, 1, 4, 4])
    cb = O.train_multi_d_adc(learn, T=4, M=4, iters=4)
    assert cb.C1.shape == (4, 4) and cb.R.shape == (4, 256, 2)
    cbl = O.train_hbpq_local(learn, cb, iters=4)
    assert cbl.Q.shape == (4, 2, 256, 2)
    # local codebooks start from the global ones and Lloyd never increases distortion
    xg = O.reconstruct(cb, *O.encode_multi_d_adc(learn, cb))
    xl = O.reconstruct_hbpq(cbl, *O.encode_hbpq(learn, cbl))
    assert ((learn - xl) ** 2).sum() <= ((learn - xg) ** 2).sum()


def test_encoding_error_literal():
    """Fig. errors' quantity by hand (literal codebooks: C^1 = [[1, 2], [3, 4]],
    C^2 = [[5, 6], [7, 8]], R_0[t] = (t, -t), R_1[t] = (2t, 1)).  x = (4, 4, 6, 5):
    first half: 13 to c^1_0, 1 to c^1_1 -> i = 1; second half: 2 to c^2_0, 10 to
    c^2_1 -> j = 0; displacement (1, 0 | 1, -1).  R_0: (t - 1)^2 + t^2 is 1 at t = 0
    and t = 1 -> the lower index 0, error 1; R_1: (2t - 1)^2 + 4 is 5 at t = 0 and
    t = 1 -> 0, error 5.  Total 6, cell 2, code (0, 0)."""
    cb = literal_codebooks()
    x = np.array([[4, 4, 6, 5]])
    cells, codes = O.encode_multi_d_adc(x, cb)
    assert cells.tolist() == [2] and codes.tolist() == [[0, 0]]
    assert O.encoding_error(cb, x).tolist() == [6.0]


def test_encoding_error_local_not_above_global_and_zero_case():
    """Local codebooks started from the global ones never encode worse (Lloyd does not
    raise distortion on their learn sets, which here are the encoded points), and a
    codebook holding every displacement encodes with zero error."""
    rng = np.random.default_rng(21)
    learn = rng.integers(0, 256, size=(3000, 8)) // np.array([1, 1, 4, 4, 1, 1, 4, 4])
    cb = O.train_multi_d_adc(learn, T=4, M=4, iters=3)
    cbl = O.train_hbpq_local(learn, cb, iters=3)
    eg = O.encoding_error(cb, learn, "global")
    el = O.encoding_error(cbl, learn, "local")
    assert el.sum() <= eg.sum() and el.sum() < eg.sum()
    from test_oracle_scoring import zero_quantization_case
    X, cbz = zero_quantization_case(0)
    assert (O.encoding_error(cbz, X) == 0).all()
