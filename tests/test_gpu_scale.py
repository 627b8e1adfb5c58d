"""Oracle parity at the target sizes, on sampled queries.

* 1B points (T = 1024, M = 8, the serving configuration): the GPU trains the
  codebooks and builds the index; the oracle takes the codebooks as given, checks
  the lists by re-encoding 20,000 sampled points (Eqs. 6-7), and searches the
  GPU's lists (copied to host memory) for 1,000 randomly sampled queries of a
  10k-query batch at L = 1k and 10k (multi-sequence traversal; a few of them also
  with the full-sort definition): identical top-100 ids and distances, hence
  identical recall.
* 100M points with M = 16 (the precision configuration): the int8 and FP16 table
  shortlists (1000, exact re-score) and the FP32 search equal the oracle's on
  200 sampled queries at L = 30k.
"""
import numpy as np
import pytest

from tests.parity import assert_topk_match

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLE = (0, 1, 17, 999, 4242, 9999)  # also checked against the full-sort traversal
BULK = tuple(sorted(np.random.default_rng(5).choice(10_000, 1_000, replace=False).tolist()))


def build(w, variant="global"):
    import torch

    import paper_1404_1831_gb300 as bpq
    import synthdata as sd
    from oracle import bpq_oracle as O
    from synthdata import device as sdev
    mix = sd.make_mixture(w.seed, w.n_comp)
    learn = sdev.points_cuda(mix, sd.STREAM_LEARN, 0, w.n_learn)
    ix = bpq.Index.train(learn, w.T, w.M, variant=variant, iters=w.kmeans_iters)
    del learn
    for s in range(0, w.n_base, 4_000_000):
        ix.add(sdev.points_cuda(mix, sd.STREAM_BASE, s, min(4_000_000, w.n_base - s)))
    ix.finalize()
    a = ix.arrays()
    cb = O.Codebooks(D=w.dim, T=w.T, M=w.M, C1=a["C1"].cpu().numpy().astype(np.int64),
                     C2=a["C2"].cpu().numpy().astype(np.int64), R=a["R"].cpu().numpy().astype(np.int64))
    lists = O.Lists(T=w.T, offsets=a["offsets"].cpu().numpy().astype(np.int64), codes=a["codes"].cpu().numpy(),
                    ids=a["ids"].cpu().numpy())
    del a
    oix = O.OracleIndex(cb=cb, lists=lists, variant="global", tables=O.fbpq_tables(cb))
    q = sdev.points_cuda(mix, sd.STREAM_QUERY, 0, w.n_query)
    torch.cuda.synchronize()
    return dict(w=w, mix=mix, ix=ix, oix=oix, q=q, qh=sd.points(mix, sd.STREAM_QUERY, 0, w.n_query))


@pytest.fixture(scope="module")
def one_b():
    import synthdata as sd
    b = build(sd.SIFT1B)
    yield b
    if "ix" in b:
        b["ix"].close()


def test_1b_sampled_reencoding(one_b):
    """20 random runs of 1000 points: the oracle's cell and codes with the index's
    codebooks equal the GPU's lists at those ids (found inside their cell: ids
    ascend within a cell)."""
    import synthdata as sd
    from oracle import bpq_oracle as O
    oix, w = one_b["oix"], one_b["w"]
    lists = oix.lists
    rng = np.random.default_rng(11)
    starts = rng.choice(w.n_base // 1000, size=20, replace=False) * 1000
    for s in starts:
        x = sd.points(one_b["mix"], sd.STREAM_BASE, int(s), 1000)
        cells, codes = O.encode_multi_d_adc(x, oix.cb)
        for j in range(1000):
            lo, hi = lists.offsets[cells[j]], lists.offsets[cells[j] + 1]
            p = lo + int(np.searchsorted(lists.ids[lo:hi], s + j))
            assert p < hi and lists.ids[p] == s + j
            assert np.array_equal(lists.codes[p], codes[j])


@pytest.mark.parametrize("L", [1_000, 10_000])
def test_1b_search_sampled(one_b, L):
    from oracle import bpq_oracle as O
    k = 100
    ids, dists = one_b["ix"].search(one_b["q"], L, k, "fbpq")
    one_b["ix"].search_status()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    exact = 0
    for n in SAMPLE:
        o_ids, o_d, _, _ = O.search_one(one_b["oix"], one_b["qh"][n], L, k, "fbpq", traversal="full_sort")
        exact += assert_topk_match(ids[n:n + 1], dists[n:n + 1], o_ids[None], o_d[None])
    assert exact == len(SAMPLE)
    exact = 0
    for n in BULK:
        o_ids, o_d, _, _ = O.search_one(one_b["oix"], one_b["qh"][n], L, k, "fbpq")
        exact += assert_topk_match(ids[n:n + 1], dists[n:n + 1], o_ids[None], o_d[None])
    assert exact == len(BULK)  # bit-identical lists on every sampled query


@pytest.fixture(scope="module")
def c3(one_b):
    import gc

    import torch

    import synthdata as sd
    if "ix" in one_b:
        one_b["ix"].close()  # the 1B index is no longer needed
    one_b.clear()
    gc.collect()
    torch.cuda.empty_cache()
    return build(sd.SIFT100M_M16)


@pytest.mark.parametrize("precision", ["int8", "fp16", "fp32"])
def test_100m_m16_shortlists_sampled(c3, precision):
    from oracle import bpq_oracle as O
    L, k, S = 30_000, 100, 1000
    if precision == "fp32":
        ids, dists = c3["ix"].search(c3["q"], L, k, "fbpq")
    else:
        ids, dists = c3["ix"].search_shortlist(c3["q"], L, k, shortlist=S, precision=precision)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    exact = 0
    picks = SAMPLE + BULK[::5]
    for n in picks:
        if precision == "fp32":
            o_ids, o_d, _, _ = O.search_one(c3["oix"], c3["qh"][n], L, k, "fbpq")
        else:
            o_ids, o_d = O.search_shortlist_one(c3["oix"], c3["qh"][n], L, k, S, precision)
        exact += assert_topk_match(ids[n:n + 1], dists[n:n + 1], o_ids[None], o_d[None])
    assert exact == len(picks)
