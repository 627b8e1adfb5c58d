"""Pins for the oracle's scorers (§2.3.3, §3.1, §3.2), ranking and recall."""
import json
import os

import numpy as np
import pytest

from oracle import bpq_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fbpq_equals_reconstruction_bit_exact(tiny_oracle):
    """Eq. 8 + Eq. 9 is an identity: FBPQ and explicit reconstruction agree
    exactly (all terms are integers below 2^53 in FP64), so recall is equal (§3.1)."""
    idx, Q = tiny_oracle["index"], tiny_oracle["queries"]
    cb, lists = idx.cb, idx.lists
    rng = np.random.default_rng(0)
    pos = rng.integers(0, len(lists.ids), size=4000)
    cell_of = np.searchsorted(lists.offsets, pos, side="right") - 1
    for q in Q[:10]:
        a = O.dist_fbpq(q, cb, idx.tables, cell_of, lists.codes[pos])
        b = O.dist_reconstruct(q, O.reconstruct(cb, cell_of, lists.codes[pos]))
        assert np.array_equal(a, b)
    ra = O.search(idx, Q[:20], 10_000, 100, "fbpq")
    rb = O.search(idx, Q[:20], 10_000, 100, "recon")
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])


def test_fbpq_with_a_dropped_term_fails(tiny_oracle):
    """A plausible mistake (dropping the 2<c^2_j, r_k> cross terms of Eq. 9) is caught."""
    idx, q = tiny_oracle["index"], tiny_oracle["queries"][0]
    cb = idx.cb
    tab = O.FbpqTables(n1=idx.tables.n1, n2=idx.tables.n2, nR=idx.tables.nR,
                       X1=idx.tables.X1, X2=np.zeros_like(idx.tables.X2))
    pos = np.arange(0, len(idx.lists.ids), 97)
    cell_of = np.searchsorted(idx.lists.offsets, pos, side="right") - 1
    a = O.dist_fbpq(q, cb, tab, cell_of, idx.lists.codes[pos])
    b = O.dist_reconstruct(q, O.reconstruct(cb, cell_of, idx.lists.codes[pos]))
    assert not np.array_equal(a, b)


def zero_quantization_case(seed, N=200, D=8, T=2):
    """Every 1-D residual value is a codeword: M = D and the residual k-means starts
    from all N <= 256 training residuals, so PQ reconstruction is exact."""
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 256, size=(N, D))
    M = D
    h = D // 2
    C1, _ = O.kmeans(X[:, :h], T, 3)
    C2, _ = O.kmeans(X[:, h:], T, 3)
    i, j = O.coarse_cells(X, C1, C2)
    disp = X - np.concatenate([C1[i], C2[j]], axis=1)
    R = np.zeros((M, O.KSUB, 1), dtype=np.int64)
    for k in range(M):
        vals = disp[:, k:k + 1]
        init = np.concatenate([vals, np.repeat(vals[-1:], O.KSUB - N, axis=0)])
        R[k] = O.kmeans(vals, O.KSUB, 2, init=init)[0]
    cb = O.Codebooks(D=D, T=T, M=M, C1=C1, C2=C2, R=R)
    return X, cb


@pytest.mark.parametrize("seed", range(5))
def test_zero_quantization_reduces_to_exact_knn(seed):
    X, cb = zero_quantization_case(seed)
    idx = O.build_index(cb, X)
    # reconstruction is exact, so ADC distances are the true distances
    xh = O.reconstruct(cb, *O.encode_multi_d_adc(X, cb))
    assert np.array_equal(xh, X.astype(np.float64))
    rng = np.random.default_rng(100 + seed)
    Q = rng.integers(0, 256, size=(10, X.shape[1]))
    ids, dists, totals = O.search(idx, Q, len(X), 10, "fbpq")
    assert (totals == len(X)).all()
    for n, q in enumerate(Q):
        true = ((X - q) ** 2).sum(1)
        order = np.lexsort((np.arange(len(X)), true))[:10]
        assert ids[n].tolist() == order.tolist()
        assert dists[n].tolist() == true[order].astype(float).tolist()
    nn = O.exact_nn(X, Q)
    assert O.recall_at(ids, nn, 1) == 1.0


def test_hbpq_with_global_copies_equals_multi_d_adc(tiny_oracle):
    """HBPQ with every local codebook equal to the global one is Multi-D-ADC."""
    cb = tiny_oracle["cb"]
    m2 = cb.M // 2
    loc = O.Codebooks(D=cb.D, T=cb.T, M=cb.M, C1=cb.C1, C2=cb.C2, R=cb.R,
                      Q=np.broadcast_to(cb.R[:m2], (cb.T,) + cb.R[:m2].shape).copy(),
                      S=np.broadcast_to(cb.R[m2:], (cb.T,) + cb.R[m2:].shape).copy())
    X = tiny_oracle["base"][:3000]
    cg, kg = O.encode_multi_d_adc(X, cb)
    cl, kl = O.encode_hbpq(X, loc)
    assert np.array_equal(cg, cl) and np.array_equal(kg, kl)
    idx = O.build_index(loc, X, variant="local")
    gidx = O.build_index(cb, X)
    q = tiny_oracle["queries"][:5]
    a = O.search(idx, q, 1000, 20, "hbpq")
    b = O.search(gidx, q, 1000, 20, "recon")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_topk_order_ties_and_padding():
    ids, d = O.topk([5.0, 1.0, 5.0, 3.0], [7, 9, 2, 4], 6)
    assert ids.tolist() == [9, 4, 2, 7, -1, -1]
    assert d.tolist()[:4] == [1.0, 3.0, 5.0, 5.0] and np.isinf(d[4:]).all()


def test_recall_and_exact_nn():
    base = np.array([[0, 0], [3, 4], [0, 0], [10, 10]])
    nn = O.exact_nn(base, np.array([[0, 1], [9, 9]]))
    assert nn.tolist() == [0, 3]  # tie between ids 0 and 2 goes to 0
    res = np.array([[2, 0, 1], [1, 2, 0]])
    assert O.recall_at(res, nn, 1) == 0.0 and O.recall_at(res, nn, 2) == 0.5
    assert O.recall_at(res, nn, 3) == 0.5


def test_memory_formulas_reproduce_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_memory.json")))
    e = g["fbpq_tables"]
    assert O.fbpq_table_floats(e["T"], e["M"], e["K"]) * 4 == e["value_mib"] * 2 ** 20
    e = g["fbpq_norms"]
    assert O.fbpq_norm_floats(e["T"], e["M"], e["K"]) * 4 < e["max_mib"] * 2 ** 20
    e = g["hbpq_sift1b_local"]
    assert O.hbpq_local_floats(e["T"], e["D"], e["K"]) * 4 == e["value_gib"] * 2 ** 30
    e = g["hbpq_gist50m_local"]
    extra = O.hbpq_local_floats(e["T"], e["D"], e["K"]) * 4 / 2 ** 30
    assert abs(extra - (e["printed_after_gb"] - e["printed_before_gb"])) < 0.01


def test_hbpq_tables_literal():
    """The regrouped HBPQ distance by hand (literal codebooks of the encode pins:
    C^1 = [[1, 2], [3, 4]], C^2 = [[5, 6], [7, 8]], Q^i_0[t] = (10 i + t, 0),
    S^j_0[t] = (0, -t - j)).  Query q = (10, 0, 5, 5), cell (1, 1), code (3, 5):
      xhat = [3 + 13, 4 + 0, 7 + 0, 8 - 6] = [16, 4, 7, 2], ||q - xhat||^2 = 36 + 16 + 4 + 9 = 65;
      d1[1] = 7^2 + 4^2 = 65, d2[1] = 2^2 + 3^2 = 13;
      A[0][3] = 13^2 + 2 (3*13 + 4*0) - 2 (10*13 + 0*0) = 169 + 78 - 260 = -13;
      B[0][5] = 6^2 + 2 (7*0 + 8*(-6)) - 2 (5*0 + 5*(-6)) = 36 - 96 + 60 = 0;
      65 + 13 - 13 + 0 = 65."""
    from test_oracle_encode import literal_codebooks
    cb = literal_codebooks()
    q = np.array([10, 0, 5, 5])
    A, B = O.hbpq_tables(q, cb, 1, 1)
    assert A[0][3] == -13.0 and B[0][5] == 0.0
    assert O.dist_hbpq_tables(q, cb, np.array([3]), np.array([[3, 5]])).tolist() == [65.0]


@pytest.fixture(scope="module")
def tiny_local(tiny_oracle):
    cb = O.train_hbpq_local(tiny_oracle["learn"], tiny_oracle["cb"], 3)
    X = tiny_oracle["base"][:20000]
    return cb, O.build_index(cb, X, variant="local")


def test_hbpq_tables_equal_reconstruction_bit_exact(tiny_oracle, tiny_local):
    """The table form is an exact regrouping of the O(D) HBPQ reconstruction
    distance (§3.2): equal bit for bit on the integer grid, and the searches agree."""
    cb, idx = tiny_local
    lists = idx.lists
    rng = np.random.default_rng(5)
    pos = rng.integers(0, len(lists.ids), size=3000)
    cell_of = np.searchsorted(lists.offsets, pos, side="right") - 1
    for q in tiny_oracle["queries"][:6]:
        a = O.dist_hbpq_tables(q, cb, cell_of, lists.codes[pos])
        b = O.dist_reconstruct(q, O.reconstruct_hbpq(cb, cell_of, lists.codes[pos]))
        assert np.array_equal(a, b)
    Q = tiny_oracle["queries"][:8]
    ra = O.search(idx, Q, 3000, 50, "hbpq_tables")
    rb = O.search(idx, Q, 3000, 50, "hbpq")
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])


def test_hbpq_tables_catch_dropped_or_swapped_terms(tiny_oracle, tiny_local):
    """Plausible mistakes in the table form differ from the reconstruction: the
    cross term 2<c^1_i|k, Q^i_k[t]> left out, or the global R_k used in place of
    the local codebooks."""
    cb, idx = tiny_local
    q = tiny_oracle["queries"][0]
    lists = idx.lists
    pos = np.arange(0, len(lists.ids), 13)
    cell_of = np.searchsorted(lists.offsets, pos, side="right") - 1
    truth = O.dist_reconstruct(q, O.reconstruct_hbpq(cb, cell_of, lists.codes[pos]))
    no_cross = O.Codebooks(D=cb.D, T=cb.T, M=cb.M, C1=np.zeros_like(cb.C1), C2=cb.C2, R=cb.R, Q=cb.Q, S=cb.S)
    i = cell_of // cb.T
    d1_true, _ = O.coarse_distances(q, cb)
    d1_zero, _ = O.coarse_distances(q, no_cross)
    # the same tables with c^1 zeroed in the cross term only: add back the true d1
    wrong = O.dist_hbpq_tables(q, no_cross, cell_of, lists.codes[pos]) - d1_zero[i] + d1_true[i]
    assert not np.array_equal(wrong, truth)
    m2 = cb.M // 2
    glob = O.Codebooks(D=cb.D, T=cb.T, M=cb.M, C1=cb.C1, C2=cb.C2, R=cb.R,
                       Q=np.broadcast_to(cb.R[:m2], cb.Q.shape).copy(),
                       S=np.broadcast_to(cb.R[m2:], cb.S.shape).copy())
    assert not np.array_equal(O.dist_hbpq_tables(q, glob, cell_of, lists.codes[pos]), truth)
