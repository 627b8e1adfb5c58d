"""Batching machinery: search graphs (one CUDA graph launch per batch) and the
autotuner's scan schedule.  Neither may change an answer: every replay equals
bpq_search of the same queries and budgets."""
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


def as_np(t):
    return [x.cpu().numpy().copy() for x in t]


@pytest.mark.parametrize("W", [0, 700])
def test_graph_replays_equal_search(gix, tiny_oracle, W):
    import synthdata as sd
    qn = sd.points(tiny_oracle["mix"], sd.STREAM_QUERY, 0, 200).astype(np.float32)
    Ls = np.array([100, 1000, 10_000, 30_000] * 25, dtype=np.int64)
    gix.set_scan_work_size(W)
    try:
        q = torch.as_tensor(qn[:100], device=DEV)
        g = gix.graph(q, Ls, 50, "fbpq")
        ref = as_np(gix.search(q, Ls, 50, "fbpq"))
        for _ in range(3):  # replays
            got = as_np(g.launch())
            torch.cuda.synchronize()
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        # new queries written into the graph's input buffer
        q.copy_(torch.as_tensor(qn[100:], device=DEV))
        got = as_np(g.launch())
        ref2 = as_np(gix.search(q, Ls, 50, "fbpq"))
        assert np.array_equal(got[0], ref2[0]) and np.array_equal(got[1], ref2[1])
        o_ids, o_d, _ = O.search(tiny_oracle["index"], qn[100:120], Ls[:20], 50, "fbpq")
        assert assert_topk_match(got[0][:20], got[1][:20], o_ids, o_d) == 20
        # new budgets, read from the graph's page-locked buffer at the next launch
        torch.cuda.synchronize()
        L2 = Ls[::-1].copy()
        g.set_budgets(L2)
        got = as_np(g.launch())
        ref3 = as_np(gix.search(q, L2, 50, "fbpq"))
        assert np.array_equal(got[0], ref3[0]) and np.array_equal(got[1], ref3[1])
        g.close()
    finally:
        gix.set_scan_work_size(0)


def test_graph_scalar_budget_and_reconstruction(gix, tiny_oracle):
    q = torch.as_tensor(tiny_oracle["queries"], dtype=torch.float32, device=DEV)
    for scorer in ("recon", "fbpq_tables"):
        g = gix.graph(q, 5000, 20, scorer)
        got = as_np(g.launch())
        ref = as_np(gix.search(q, 5000, 20, scorer))
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        with pytest.raises(Exception):
            g.set_budgets(np.full(len(q), 100))  # captured with one budget for every query
        g.close()


def test_autotune_keeps_answers(gix, tiny_oracle):
    q = torch.as_tensor(tiny_oracle["queries"], dtype=torch.float32, device=DEV)
    Ls = np.array([50_000] * 50 + [300] * 50, dtype=np.int64)
    ref = as_np(gix.search(q, Ls, 100, "fbpq"))
    W = gix.autotune(q, Ls, 100, "fbpq")
    assert W in (0, 4096, 8192, 16384, 32768)
    got = as_np(gix.search(q, Ls, 100, "fbpq"))  # the tuned class's schedule
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    g = gix.graph(q, Ls, 100, "fbpq")  # a graph captures the tuned schedule
    got = as_np(g.launch())
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    g.close()


def test_graph_hbpq(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    learn = torch.as_tensor(t["learn"], dtype=torch.float32, device=DEV)
    ix = bpq.Index.train(learn, t["w"].T, t["w"].M, variant="local", iters=4)
    ix.add(torch.as_tensor(t["base"][:40_000], dtype=torch.float32, device=DEV))
    ix.finalize()
    q = torch.as_tensor(t["queries"], dtype=torch.float32, device=DEV)
    Ls = np.array([300, 4000, 40_000, 20] * 25, dtype=np.int64)
    g = ix.graph(q, Ls, 100, "hbpq")
    got = as_np(g.launch())
    ref = as_np(ix.search(q, Ls, 100, "hbpq"))
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    g.close()
