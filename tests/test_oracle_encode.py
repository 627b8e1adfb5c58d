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


def test_reconstruct_is_equation_7():
    rng = np.random.default_rng(12)
    cb = small_codebooks(rng)
    cell = np.array([1 * 4 + 3])
    code = np.array([[5, 6, 7, 8]])
    xh = O.reconstruct(cb, cell, code)[0]
    expect = np.concatenate([cb.C1[1], cb.C2[3]]) + np.concatenate([cb.R[k][code[0, k]] for k in range(4)])
    assert np.array_equal(xh, expect)


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
