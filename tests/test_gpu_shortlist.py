"""GPU parity of the reduced-precision shortlist search (bpq_search_shortlist, int8 and
FP16 tables) and of the M = 16 scans against the oracle, on the tiny workload (100k
points, T = 64)."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _gpu_index(cb, base):
    import paper_1404_1831_gb300 as bpq
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    ix.add(torch.as_tensor(base, dtype=torch.float32, device=DEV))
    ix.finalize()
    return ix


@pytest.fixture(scope="module")
def m8(tiny_oracle):
    t = tiny_oracle
    return dict(ix=_gpu_index(t["cb"], t["base"]), index=t["index"], qh=t["queries"],
                q=torch.as_tensor(t["queries"], dtype=torch.float32, device=DEV))


@pytest.fixture(scope="module")
def m16(tiny_oracle):
    t = tiny_oracle
    w = t["w"]
    cb = O.train_multi_d_adc(t["learn"], w.T, 16, w.kmeans_iters)
    index = O.build_index(cb, t["base"])
    return dict(ix=_gpu_index(cb, t["base"]), index=index, qh=t["queries"][:40],
                q=torch.as_tensor(t["queries"][:40], dtype=torch.float32, device=DEV))


def _check(fx, L, k, S, nq=None, precision="int8"):
    nq = nq or len(fx["qh"])
    ids, dists = fx["ix"].search_shortlist(fx["q"][:nq], L, k, shortlist=S, precision=precision)
    o_ids, o_d = O.search_shortlist(fx["index"], fx["qh"][:nq], L, k, S, precision)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    assert np.array_equal(ids, o_ids), "shortlist ids differ"
    assert np.array_equal(dists.astype(np.float64), o_d), "shortlist distances differ"
    return ids, dists


@pytest.mark.parametrize("precision", ["int8", "fp16"])
@pytest.mark.parametrize("L,k,S", [(10_000, 100, 1000), (3_000, 10, 100), (10_000, 100, 100), (20_000, 1, 1024)])
def test_shortlist_matches_oracle_m8(m8, L, k, S, precision):
    _check(m8, L, k, S, nq=40, precision=precision)


def test_shortlist_pads_when_few_candidates(m8):
    ids, dists = _check(m8, 1, 100, 1000, nq=10)
    assert (ids == -1).any() and np.isinf(dists).any()


def test_full_shortlist_equals_fbpq_search(m8):
    """A shortlist as long as the candidate list (L' < 1024 at L = 500) returns the
    FP32 FBPQ search's lists."""
    a = [t.cpu().numpy() for t in m8["ix"].search(m8["q"], 500, 50, "fbpq")]
    b = [t.cpu().numpy() for t in m8["ix"].search_shortlist(m8["q"], 500, 50, shortlist=1024)]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_fbpq_and_reconstruction_match_oracle_m16(m16):
    for scorer, o_scorer in (("fbpq", "fbpq"), ("fbpq_tables", "fbpq"), ("recon", "recon")):
        ids, dists = m16["ix"].search(m16["q"], 5_000, 50, scorer)
        o_ids, o_d, _ = O.search(m16["index"], m16["qh"], 5_000, 50, o_scorer)
        exact = assert_topk_match(ids.cpu().numpy(), dists.cpu().numpy(), o_ids, o_d)
        assert exact == len(o_ids)


@pytest.mark.parametrize("precision", ["int8", "fp16"])
def test_shortlist_matches_oracle_m16(m16, precision):
    _check(m16, 10_000, 100, 1000, precision=precision)


def test_fp16_short_shortlist_ranks_like_the_oracle(m8):
    """A shortlist much shorter than the candidate list (S = k = 10) depends on the
    FP16 scores themselves, not only on the exact re-score."""
    _check(m8, 10_000, 10, 10, nq=40, precision="fp16")


def test_shortlist_rejects_bad_arguments(m8):
    import paper_1404_1831_gb300 as bpq
    for k, S in ((100, 50), (10, 1025), (0, 10)):
        with pytest.raises(bpq.BpqError):
            m8["ix"].search_shortlist(m8["q"][:2], 1000, k, shortlist=S)


@pytest.mark.parametrize("precision", ["int8", "fp16"])
def test_shortlist_cut_inside_a_large_tie_group(tiny_oracle, precision):
    """4000 copies of one point under distinct ids share a cell, a code and a score: a
    shortlist of 1000 is cut inside that tie group, by list position as in the oracle
    (the group is larger than the scan's block buffer keeps by score alone)."""
    import paper_1404_1831_gb300 as bpq
    cb = tiny_oracle["cb"]
    base = tiny_oracle["base"][:6000]
    X = np.concatenate([base, np.repeat(base[:1], 4000, axis=0)])
    ids = np.arange(len(X), dtype=np.int32)
    oix = O.build_index(cb, X, ids=ids)
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    ix.add(torch.as_tensor(X, dtype=torch.float32, device=DEV), ids=torch.as_tensor(ids, device=DEV))
    ix.finalize()
    qn = np.concatenate([base[:1].astype(np.float64), base[:1] + 0.5, tiny_oracle["queries"][:2]])
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    g_ids, g_d = [t.cpu().numpy() for t in ix.search_shortlist(q, 5000, 100, shortlist=1000, precision=precision)]
    o_ids, o_d = O.search_shortlist(oix, qn, 5000, 100, 1000, precision)
    assert np.array_equal(g_ids, o_ids)
    assert np.array_equal(g_d.astype(np.float64), o_d)
    copies = np.r_[0, 6000:10000]  # base[0] and its copies
    assert np.isin(g_ids[0], copies).sum() >= 90  # the tie group fills the first answer
