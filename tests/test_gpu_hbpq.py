"""GPU parity for HBPQ (§3.2): local codebook training, local encoding and the
HBPQ scorer against the FP64 oracle, on a reduced tiny workload."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hbpq(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    w = t["w"]
    iters = 4
    cb = O.train_multi_d_adc(t["learn"], w.T, w.M, iters)
    cbl = O.train_hbpq_local(t["learn"], cb, iters)
    base = t["base"][:40_000]
    oix = O.build_index(cbl, base, variant="local")
    learn = torch.as_tensor(t["learn"], dtype=torch.float32, device=DEV)
    ix = bpq.Index.train(learn, w.T, w.M, variant="local", iters=iters)
    ix.add(torch.as_tensor(base, dtype=torch.float32, device=DEV))
    ix.finalize()
    return dict(ix=ix, oix=oix, cbl=cbl, base=base)


def test_local_training_bit_exact(hbpq):
    a = hbpq["ix"].arrays()
    assert np.array_equal(a["Q"].cpu().numpy(), hbpq["cbl"].Q.astype(np.float32))
    assert np.array_equal(a["S"].cpu().numpy(), hbpq["cbl"].S.astype(np.float32))


def test_local_encoding_bit_exact(hbpq):
    a = hbpq["ix"].arrays()
    assert np.array_equal(a["codes"].cpu().numpy(), hbpq["oix"].lists.codes)
    assert np.array_equal(a["offsets"].cpu().numpy().astype(np.int64), hbpq["oix"].lists.offsets)


def test_hbpq_search_matches_oracle(hbpq, tiny_oracle):
    qn = tiny_oracle["queries"][:40]
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    ids, d = hbpq["ix"].search(q, 4000, 50, "hbpq")
    o_ids, o_d, _ = O.search(hbpq["oix"], qn, 4000, 50, "hbpq")
    assert assert_topk_match(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d) == len(qn)


def search_both(hbpq, qn, L, k, scorer="hbpq"):
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    ids, d = hbpq["ix"].search(q, L, k, scorer)
    hbpq["ix"].search_status()
    o_ids, o_d, _ = O.search(hbpq["oix"], qn, L, k, "hbpq_tables")
    return ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d


@pytest.mark.parametrize("L", [1, 300, 4000, 40_000])
@pytest.mark.parametrize("k", [1, 37, 128])
def test_hbpq_table_form_matches_oracle(hbpq, tiny_oracle, L, k):
    """Per-(query, half-cell) tables on the tensor cores + M-lookup scan (§3.2 regrouped):
    identical top-k to the oracle's table form (itself pinned equal to the O(D)
    reconstruction), from a single cell (L = 1) to every cell of the index."""
    qn = tiny_oracle["queries"][:24]
    ids, d, o_ids, o_d = search_both(hbpq, qn, L, k)
    assert assert_topk_match(ids, d, o_ids, o_d) == len(qn)


def test_hbpq_uneven_budgets_and_reconstruction_scorer(hbpq, tiny_oracle):
    """Per-query budgets in one batch; the table form equals the paper's O(D) form
    (scorer hbpq_recon) bit for bit."""
    qn = tiny_oracle["queries"][:60]
    Ls = np.array([1, 10, 100, 1000, 10_000, 40_000] * 10, dtype=np.int64)
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    a = [t.cpu().numpy() for t in hbpq["ix"].search(q, Ls, 100, "hbpq")]
    b = [t.cpu().numpy() for t in hbpq["ix"].search(q, Ls, 100, "hbpq_recon")]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    o_ids, o_d, _ = O.search(hbpq["oix"], qn, Ls, 100, "hbpq")
    assert assert_topk_match(a[0], a[1], o_ids, o_d) == len(qn)


def test_hbpq_large_k_uses_reconstruction(hbpq, tiny_oracle):
    """k > 128 takes the O(D) scan: still identical to the oracle."""
    qn = tiny_oracle["queries"][:10]
    ids, d, o_ids, o_d = search_both(hbpq, qn, 4000, 300)
    assert assert_topk_match(ids, d, o_ids, o_d) == len(qn)


def test_hbpq_table_overflow_falls_back(hbpq, tiny_oracle):
    """With a table budget too small for most queries, the queries that do not fit
    are scored by the O(D) reconstruction scan: the answers do not change."""
    qn = tiny_oracle["queries"][:32]
    ix = hbpq["ix"]
    ref = search_both(hbpq, qn, 20_000, 100)
    try:
        ix.set_hbpq_table_budget(3.0)  # 96 slots for 32 queries that need ~100 each
        got = search_both(hbpq, qn, 20_000, 100)
    finally:
        ix.set_hbpq_table_budget(0.0)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    assert assert_topk_match(got[0], got[1], got[2], got[3]) == len(qn)


def test_hbpq_chunked_workspace(hbpq, tiny_oracle):
    """A workspace for a few queries processes the batch in chunks, tables included."""
    import paper_1404_1831_gb300 as bpq
    qn = tiny_oracle["queries"][:40]
    ix = hbpq["ix"]
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    need = bpq.lib().bpq_search_workspace_size(ix._h, 3, 4000, 50, bpq.SCORERS["hbpq"])
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    ids, d = ix.search(q, 4000, 50, "hbpq", workspace=ws)
    o_ids, o_d, _ = O.search(hbpq["oix"], qn, 4000, 50, "hbpq")
    assert assert_topk_match(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d) == len(qn)


def test_encoding_error_matches_oracle(hbpq, tiny_oracle):
    """Fig. errors' per-point squared encoding error on the GPU equals the oracle's,
    bit for bit (integer grid), for the local codebooks and the global ones.  (Which
    is lower depends on the data: with 20k learn points over 64 half-cells the local
    codebooks have about 300 points for 256 codewords and do not generalize.)"""
    import paper_1404_1831_gb300 as bpq
    X = tiny_oracle["base"][:20_000]
    x = torch.as_tensor(X, dtype=torch.float32, device=DEV)
    got = hbpq["ix"].encoding_error(x).cpu().numpy()
    assert np.array_equal(got.astype(np.float64), O.encoding_error(hbpq["cbl"], X, "local"))
    cb = O.train_multi_d_adc(tiny_oracle["learn"], hbpq["cbl"].T, hbpq["cbl"].M, 4)
    g = bpq.Index.create(cb.C1, cb.C2, cb.R)
    got_g = g.encoding_error(x).cpu().numpy()
    assert np.array_equal(got_g.astype(np.float64), O.encoding_error(cb, X, "global"))
