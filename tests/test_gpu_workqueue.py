"""Persistent work-queue scan (bpq_set_scan_work_size): queries cut into work items
of about W candidates, partial top-k lists merged by (distance, id).  The answers
must equal the one-CTA-per-query scan bit for bit, and the oracle's."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def gix(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    cb = tiny_oracle["cb"]
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    ix.add(torch.as_tensor(tiny_oracle["base"], dtype=torch.float32, device=DEV))
    ix.finalize()
    return ix


def both(ix, q, L, k, scorer, W):
    ix.set_scan_work_size(0)
    a = [t.cpu().numpy() for t in ix.search(q, L, k, scorer)]
    try:
        ix.set_scan_work_size(W)
        b = [t.cpu().numpy() for t in ix.search(q, L, k, scorer)]
        ix.search_status()
    finally:
        ix.set_scan_work_size(0)
    return a, b


@pytest.mark.parametrize("W", [300, 2000, 50_000])
@pytest.mark.parametrize("k", [1, 50, 128])
def test_work_queue_equals_per_query_fbpq(gix, tiny_oracle, W, k):
    qn = tiny_oracle["queries"]
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    Ls = np.array([1, 10, 300, 3000, 30_000, 100_000] * 17, dtype=np.int64)[:len(qn)]
    a, b = both(gix, q, Ls, k, "fbpq", W)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    o_ids, o_d, _ = O.search(tiny_oracle["index"], qn[:30], Ls[:30], k, "fbpq")
    assert assert_topk_match(b[0][:30], b[1][:30], o_ids, o_d) == 30


def test_work_queue_hbpq(tiny_oracle):
    """The HBPQ table form through the work queue (items of queries whose tables
    did not fit are not built: the O(D) fallback answers them)."""
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    w = t["w"]
    learn = torch.as_tensor(t["learn"], dtype=torch.float32, device=DEV)
    ix = bpq.Index.train(learn, w.T, w.M, variant="local", iters=4)
    ix.add(torch.as_tensor(t["base"][:40_000], dtype=torch.float32, device=DEV))
    ix.finalize()
    q = torch.as_tensor(t["queries"], dtype=torch.float32, device=DEV)
    Ls = np.array([100, 4000, 40_000, 7] * 25, dtype=np.int64)
    a, b = both(ix, q, Ls, 100, "hbpq", 700)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ix.set_hbpq_table_budget(3.0)  # most queries fall back to the O(D) scan
    try:
        a2, b2 = both(ix, q, Ls, 100, "hbpq", 700)
    finally:
        ix.set_hbpq_table_budget(0.0)
    assert np.array_equal(a[0], b2[0]) and np.array_equal(a[1], b2[1])


def test_work_queue_empty_index_and_tiny_batches(gix, tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    cb = tiny_oracle["cb"]
    empty = bpq.Index.create(cb.C1, cb.C2, cb.R)
    empty.finalize()
    q = torch.as_tensor(tiny_oracle["queries"][:3], dtype=torch.float32, device=DEV)
    empty.set_scan_work_size(100)
    ids, d = empty.search(q, 1000, 10, "fbpq")
    assert (ids.cpu().numpy() == -1).all() and np.isinf(d.cpu().numpy()).all()
    a, b = both(gix, q[:1], 50_000, 100, "fbpq", 200)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
