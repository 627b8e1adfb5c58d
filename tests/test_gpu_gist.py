"""GIST-shaped parity (D = 384, M = 8, so D/2 = 192 and D/M = 48): the shape of the
paper's GIST50M rows (Table FBPQ, Table gist_performance), on a small synthetic case.
Training, encoding, lists, query tables and the FBPQ / paper-table / reconstruction
/ HBPQ searches against the FP64 oracle."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def gist():
    import paper_1404_1831_gb300 as bpq
    import synthdata as sd
    w = sd.TINY_GIST
    mix = sd.make_mixture(w.seed, w.n_comp, w.dim)
    learn = sd.points(mix, sd.STREAM_LEARN, 0, w.n_learn)
    base = sd.points(mix, sd.STREAM_BASE, 0, w.n_base)
    queries = sd.points(mix, sd.STREAM_QUERY, 0, w.n_query)
    cb = O.train_multi_d_adc(learn, w.T, w.M, w.kmeans_iters)
    oix = O.build_index(cb, base)
    lt = torch.as_tensor(learn, dtype=torch.float32, device=DEV)
    ix = bpq.Index.train(lt, w.T, w.M, iters=w.kmeans_iters)
    ix.add(torch.as_tensor(base, dtype=torch.float32, device=DEV))
    ix.finalize()
    return dict(w=w, learn=learn, base=base, queries=queries, cb=cb, oix=oix, ix=ix, lt=lt)


def test_gist_training_and_lists_bit_exact(gist):
    a = gist["ix"].arrays()
    for name in ("C1", "C2", "R"):
        assert np.array_equal(a[name].cpu().numpy(), getattr(gist["cb"], name).astype(np.float32)), name
    lists = gist["oix"].lists
    assert np.array_equal(a["offsets"].cpu().numpy().astype(np.int64), lists.offsets)
    assert np.array_equal(a["codes"].cpu().numpy(), lists.codes)


def test_gist_query_tables_exact(gist):
    """Coarse tables with K = 192 on the tensor cores (12 MMA K-steps) and the PQ table
    with K = 48, equal to the oracle's FP64 values."""
    q = torch.as_tensor(gist["queries"], dtype=torch.float32, device=DEV)
    d1, d2, lut = [t.cpu().numpy() for t in gist["ix"].query_tables(q)]
    for n, qv in enumerate(gist["queries"]):
        o1, o2 = O.coarse_distances(qv, gist["cb"])
        assert np.array_equal(d1[n], o1) and np.array_equal(d2[n], o2)
        assert np.array_equal(lut[n], O.pq_table(qv, gist["cb"]))


@pytest.mark.parametrize("L", [500, 5_000, 60_000])
@pytest.mark.parametrize("scorer", ["fbpq", "fbpq_tables", "recon"])
def test_gist_search_matches_oracle(gist, L, scorer):
    qn = gist["queries"]
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    ids, d = gist["ix"].search(q, L, 50, scorer)
    o_ids, o_d, _ = O.search(gist["oix"], qn, L, 50, "fbpq")
    assert assert_topk_match(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d) == len(qn)


def test_gist_hbpq_matches_oracle(gist):
    """HBPQ with D/M = 48: local training bit-exact, the table form (tabulated on the
    CUDA cores for this width) and the O(D) form equal to the oracle."""
    import paper_1404_1831_gb300 as bpq
    w = gist["w"]
    cbl = O.train_hbpq_local(gist["learn"], gist["cb"], w.kmeans_iters)
    oix = O.build_index(cbl, gist["base"], variant="local")
    ix = bpq.Index.train(gist["lt"], w.T, w.M, variant="local", iters=w.kmeans_iters)
    ix.add(torch.as_tensor(gist["base"], dtype=torch.float32, device=DEV))
    ix.finalize()
    a = ix.arrays()
    assert np.array_equal(a["Q"].cpu().numpy(), cbl.Q.astype(np.float32))
    assert np.array_equal(a["S"].cpu().numpy(), cbl.S.astype(np.float32))
    qn = gist["queries"]
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    o_ids, o_d, _ = O.search(oix, qn, 5_000, 50, "hbpq")
    for scorer in ("hbpq", "hbpq_recon"):
        ids, d = ix.search(q, 5_000, 50, scorer)
        assert assert_topk_match(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d) == len(qn)
