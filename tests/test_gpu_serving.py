"""Continuous batching (bpq_server_*): every query's answer is the same when it is
served alone and when it is served in a mix of overlapping batches with other
queries and other budgets, and batches really overlap (several in flight)."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
K = 50


@pytest.fixture(scope="module")
def served(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    import synthdata as sd
    cb = tiny_oracle["cb"]
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    ix.add(torch.as_tensor(tiny_oracle["base"], dtype=torch.float32, device=DEV))
    ix.finalize()
    qn = sd.points(tiny_oracle["mix"], sd.STREAM_QUERY, 0, 400).astype(np.float32)
    Ls = np.random.default_rng(5).choice([100, 1000, 10_000], size=len(qn)).astype(np.int64)
    alone = []
    for n in range(len(qn)):  # each query searched by itself
        i, d = ix.search(torch.as_tensor(qn[n:n + 1], device=DEV), int(Ls[n]), K, "fbpq")
        alone.append((i.cpu().numpy()[0], d.cpu().numpy()[0]))
    return dict(ix=ix, qn=qn, Ls=Ls, alone_ids=np.stack([a[0] for a in alone]),
                alone_d=np.stack([a[1] for a in alone]))


@pytest.mark.parametrize("group", [True, False])
def test_trace_answers_equal_alone(served, group):
    from paper_1404_1831_gb300 import serving
    qn, Ls = served["qn"], served["Ls"]
    arr = serving.poisson_arrivals(len(qn), 400_000.0, 9)  # 400 queries in about 1 ms
    res = serving.serve_continuous(served["ix"], qn, Ls, arr, k=K, slots=3, max_batch=32, group_by_budget=group)
    assert np.array_equal(res.ids, served["alone_ids"])
    assert np.array_equal(res.dists, served["alone_d"])
    assert (res.latency_s > 0).all()
    st = res.stats
    assert st["queries"] == len(qn) and st["batches"] >= len(qn) // 32
    assert st["max_in_flight"] >= 2  # a batch was launched while another was on the GPU


def test_answers_match_oracle(served, tiny_oracle):
    from paper_1404_1831_gb300 import serving
    qn, Ls = served["qn"][:60], served["Ls"][:60]
    res = serving.serve_continuous(served["ix"], qn, Ls, np.zeros(len(qn)), k=K, slots=2, max_batch=16)
    o_ids, o_d, _ = O.search(tiny_oracle["index"], qn, Ls, K, "fbpq")
    assert assert_topk_match(res.ids, res.dists, o_ids, o_d) == len(qn)


def test_admission_by_device_memory(served):
    """With a device budget that holds 8 queries at L = 10k per slot, no batch of
    L = 10k requests is larger than that, while L = 100 requests batch more."""
    import paper_1404_1831_gb300 as bpq
    from paper_1404_1831_gb300 import serving
    ix = served["ix"]
    per8 = bpq.lib().bpq_search_workspace_size(ix._h, 8, 10_000, K, bpq.SCORERS["fbpq"])
    srv = serving.Server(ix, k=K, slots=2, max_batch=64, L_max=10_000, device_bytes=2 * per8)
    try:
        qn = served["qn"][:64]
        srv.submit(qn, 10_000)
        srv.progress()
        assert srv.stats()["queries"] <= 16  # two slots of at most eight queries
        got = {}
        while len(got) < 64:
            srv.progress(wait=True)
            r, i, d, lat = srv.take()
            for j in range(len(r)):
                got[int(r[j])] = (i[j], d[j])
        st = srv.stats()
        assert st["batches"] >= 8
        ids = np.stack([got[n][0] for n in range(64)])
        ref = [t.cpu().numpy() for t in ix.search(torch.as_tensor(qn, device=DEV), 10_000, K, "fbpq")]
        assert np.array_equal(ids, ref[0])
        first = srv.submit(served["qn"][:64], 100)
        srv.progress()
        assert srv.stats()["batches"] - st["batches"] <= 2  # L = 100: 64 queries fit one batch per slot
        done = 0
        while done < 64:
            srv.progress(wait=True)
            done += len(srv.take()[0])
        assert first == 64
    finally:
        srv.close()
