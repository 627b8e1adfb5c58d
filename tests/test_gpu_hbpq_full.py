"""HBPQ parity on a T = 1024 index (1,048,576 cells), on sampled queries.

The GPU trains the global and local codebooks (§2.3.1, §3.2) and builds the
lists of 4M points.  The oracle takes those codebooks as given and checks the
index by re-encoding a random sample of the points (Eq. 12); it then searches the
GPU's lists with the O(D) HBPQ reconstruction distance, and the GPU's table-form
answers for a 2000-query batch must equal it on sampled queries.
"""
import numpy as np
import pytest

from tests.parity import assert_topk_match

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_BASE, N_LEARN, ITERS, NQ = 4_000_000, 1_024_000, 4, 2000
SAMPLE = (0, 1, 2, 777, 1500, 1999)


@pytest.fixture(scope="module")
def big():
    import torch

    import paper_1404_1831_gb300 as bpq
    import synthdata as sd
    from oracle import bpq_oracle as O
    from synthdata import device as sdev
    w = sd.SIFT100M
    mix = sd.make_mixture(w.seed, w.n_comp)
    learn = sdev.points_cuda(mix, sd.STREAM_LEARN, 0, N_LEARN)
    ix = bpq.Index.train(learn, w.T, w.M, variant="local", iters=ITERS)
    del learn
    for s in range(0, N_BASE, 2_000_000):
        ix.add(sdev.points_cuda(mix, sd.STREAM_BASE, s, min(2_000_000, N_BASE - s)))
    ix.finalize()
    a = {k: (v.cpu().numpy() if v is not None else None) for k, v in ix.arrays().items()}
    cb = O.Codebooks(D=w.dim, T=w.T, M=w.M, C1=a["C1"].astype(np.int64), C2=a["C2"].astype(np.int64),
                     R=a["R"].astype(np.int64), Q=a["Q"].astype(np.int64), S=a["S"].astype(np.int64))
    lists = O.Lists(T=w.T, offsets=a["offsets"].astype(np.int64), codes=a["codes"],
                    ids=a["ids"].astype(np.int64))
    oix = O.OracleIndex(cb=cb, lists=lists, variant="local")
    q = sdev.points_cuda(mix, sd.STREAM_QUERY, 0, NQ)
    torch.cuda.synchronize()
    return dict(w=w, mix=mix, ix=ix, oix=oix, q=q, qh=sd.points(mix, sd.STREAM_QUERY, 0, NQ))


def test_sampled_reencoding_matches_lists(big):
    """Cells and local codes of 20,000 points (20 random runs of 1000), re-encoded by the oracle with the
    index's codebooks, equal what the GPU stored for those ids (Eq. 12)."""
    import synthdata as sd
    from oracle import bpq_oracle as O
    rng = np.random.default_rng(3)
    starts = np.sort(rng.choice(N_BASE // 1000, size=20, replace=False)) * 1000
    ids = np.concatenate([np.arange(s, s + 1000) for s in starts])
    x = np.concatenate([sd.points(big["mix"], sd.STREAM_BASE, int(s), 1000) for s in starts])
    cells, codes = O.encode_hbpq(x, big["oix"].cb)
    lists = big["oix"].lists
    pos_of = np.empty(N_BASE, dtype=np.int64)
    pos_of[lists.ids] = np.arange(N_BASE)
    pos = pos_of[ids]
    cell_of = np.searchsorted(lists.offsets, pos, side="right") - 1
    assert np.array_equal(cell_of, cells)
    assert np.array_equal(lists.codes[pos], codes)


@pytest.mark.parametrize("L", [1_000, 30_000])
def test_hbpq_table_form_sampled(big, L):
    from oracle import bpq_oracle as O
    k = 100
    ids, dists = big["ix"].search(big["q"], L, k, "hbpq")
    big["ix"].search_status()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    exact = 0
    for n in SAMPLE:
        o_ids, o_d, _, _ = O.search_one(big["oix"], big["qh"][n], L, k, "hbpq", traversal="full_sort")
        exact += assert_topk_match(ids[n:n + 1], dists[n:n + 1], o_ids[None], o_d[None])
    assert exact == len(SAMPLE)


def test_hbpq_table_form_equals_reconstruction_batch(big):
    """The whole 2000-query batch: the table form and the O(D) form agree bit for bit."""
    a = [t.cpu().numpy() for t in big["ix"].search(big["q"], 10_000, 100, "hbpq")]
    b = [t.cpu().numpy() for t in big["ix"].search(big["q"], 10_000, 100, "hbpq_recon")]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
