"""Point shards on the GPU (the layout for an index larger than one GPU), run here as
several shard indexes on one GPU, one after the other (no kernel waits on another).

Each shard holds one id range of the points and is given the whole index's per-cell
counts (bpq_set_global_counts); its traversal then visits exactly the cells, and
reports exactly the L', of the whole index (§2.3.3), and it scores only its own
points.  Merging the shards' k best by (distance, id) must give the whole index's
lists bit for bit, for every scorer."""
import numpy as np
import pytest

from paper_1404_1831_gb300 import multi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def shards(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    cb = tiny_oracle["cb"]
    base = tiny_oracle["base"]
    n = len(base)
    full = bpq.Index.create(cb.C1, cb.C2, cb.R)
    full.add(torch.as_tensor(base, dtype=torch.float32, device=DEV))
    full.finalize()
    parts = []
    for r in range(3):
        s, c = multi.shard_points(n, r, 3)
        ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
        ix.add(torch.as_tensor(base[s:s + c], dtype=torch.float32, device=DEV),
               ids=torch.arange(s, s + c, dtype=torch.int32, device=DEV))
        ix.finalize()
        parts.append(ix)
    counts = sum(ix.cell_counts() for ix in parts)
    assert np.array_equal(counts, full.cell_counts())
    for ix in parts:
        ix.set_global_counts(counts)
    q = torch.as_tensor(tiny_oracle["queries"], dtype=torch.float32, device=DEV)
    return full, parts, q


def _merged(parts, fn, k):
    outs = [fn(ix) for ix in parts]
    return multi.merge_topk(np.stack([o[0].cpu().numpy() for o in outs]),
                            np.stack([o[1].cpu().numpy() for o in outs]), k)


@pytest.mark.parametrize("scorer", ["fbpq", "fbpq_tables", "recon"])
@pytest.mark.parametrize("L", [1, 700, 10_000, 250_000])
def test_shards_merge_to_the_whole_index_answer(shards, scorer, L):
    full, parts, q = shards
    k = 100
    a_i, a_d = [t.cpu().numpy() for t in full.search(q, L, k, scorer)]
    m_i, m_d = _merged(parts, lambda ix: ix.search(q, L, k, scorer), k)
    assert np.array_equal(a_i, m_i)
    assert np.array_equal(a_d.astype(np.float64), m_d)


def test_shards_report_the_whole_index_budget(shards):
    """Every shard visits the same cells with the same L' as the whole index."""
    full, parts, q = shards
    cap = int(full.info().n_nonempty)
    _, fn, fp = full.traverse(q, 10_000, cap)
    for ix in parts:
        _, n, p = ix.traverse(q, 10_000, cap)
        assert torch.equal(p, fp)
        assert (n <= fn).all()


def test_shard_shortlists_are_sandwiched(shards):
    """Shortlists do not split exactly: each shard keeps its own 500 best scores, so the
    union of the shards' shortlists holds the whole index's shortlist (its order within a
    shard is the whole index's order restricted to the shard) and possibly more points.
    The merged answer is therefore, rank by rank, at least as close as the whole index's
    shortlist answer and no closer than the exact FP32 search."""
    full, parts, q = shards
    k = 50
    _, w_d = [t.cpu().numpy() for t in full.search_shortlist(q, 10_000, k, shortlist=500)]
    _, e_d = [t.cpu().numpy() for t in full.search(q, 10_000, k, "fbpq")]
    m_i, m_d = _merged(parts, lambda ix: ix.search_shortlist(q, 10_000, k, shortlist=500), k)
    assert (m_d <= w_d.astype(np.float64)).all()
    assert (e_d.astype(np.float64) <= m_d).all()
    assert (m_i >= 0).all()


def test_global_counts_are_checked(shards):
    import paper_1404_1831_gb300 as bpq
    full, parts, q = shards
    c = parts[0].cell_counts()
    bad = c.copy()
    j = int(np.argmax(bad))
    bad[j] -= 1  # below the shard's own count of that cell
    with pytest.raises(bpq.BpqError):
        parts[0].set_global_counts(bad)
    with pytest.raises(ValueError):
        parts[0].set_global_counts(c[:-1])
    # without the whole index's counts a shard stops at its own L' (a different answer)
    ix = parts[1]
    ix.set_global_counts(None)
    alone = ix.search(q, 10_000, 10, "fbpq")[0]
    ix.set_global_counts(sum(p.cell_counts() for p in parts))
    shard = ix.search(q, 10_000, 10, "fbpq")[0]
    assert not torch.equal(alone, shard)


@pytest.mark.parametrize("scorer", ["hbpq", "hbpq_recon"])
def test_hbpq_shards_merge_to_the_whole_index_answer(tiny_oracle, scorer):
    """HBPQ (local codebooks, §3.2) on point shards: the per-half-cell tables are built for the
    cells every shard visits with the whole index's counts; merged = the whole index's lists."""
    import paper_1404_1831_gb300 as bpq
    from oracle import bpq_oracle as O
    t = tiny_oracle
    cbl = O.train_hbpq_local(t["learn"], t["cb"], t["w"].kmeans_iters)
    base = t["base"]
    n = len(base)

    def make(lo, cnt):
        ix = bpq.Index.create(cbl.C1, cbl.C2, cbl.R, Q=cbl.Q, S=cbl.S)
        ix.add(torch.as_tensor(base[lo:lo + cnt], dtype=torch.float32, device=DEV),
               ids=torch.arange(lo, lo + cnt, dtype=torch.int32, device=DEV))
        ix.finalize()
        return ix

    full = make(0, n)
    parts = [make(*multi.shard_points(n, r, 2)) for r in range(2)]
    counts = sum(ix.cell_counts() for ix in parts)
    for ix in parts:
        ix.set_global_counts(counts)
    q = torch.as_tensor(t["queries"], dtype=torch.float32, device=DEV)
    k = 50
    a_i, a_d = [x.cpu().numpy() for x in full.search(q, 5_000, k, scorer)]
    m_i, m_d = _merged(parts, lambda ix: ix.search(q, 5_000, k, scorer), k)
    assert np.array_equal(a_i, m_i)
    assert np.array_equal(a_d.astype(np.float64), m_d)
