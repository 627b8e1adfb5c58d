"""Parity at the full 10M-point workload (T = 1024, M = 8), on sampled queries.

The oracle trains the codebooks (4 Lloyd iterations on 100k learn points) and
encodes all 10M points in a pool of spawned processes; the GPU index is created
from those codebooks and fed the same points from the device generator.  The
lists must then agree bit for bit, and the GPU's answers for a 10k-query batch
(the launch the benchmark times) must equal the oracle's on sampled queries at
L = 1k, 10k and 100k.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from tests.parity import assert_topk_match

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

LEARN, ITERS, CHUNK = 100_000, 4, 250_000
SAMPLE = (0, 1, 2, 3, 1234, 4321, 7777, 9999)


def _encode_chunk(task):
    import synthdata as sd
    from oracle import bpq_oracle as O
    seed, n_comp, start, count, cb = task
    x = sd.points(sd.make_mixture(seed, n_comp), sd.STREAM_BASE, start, count)
    return O.encode_multi_d_adc(x, cb)


@pytest.fixture(scope="module")
def full():
    import torch

    import paper_1404_1831_gb300 as bpq
    import synthdata as sd
    from oracle import bpq_oracle as O
    from synthdata import device as sdev
    w = sd.SIFT10M
    mix = sd.make_mixture(w.seed, w.n_comp)
    cb = O.train_multi_d_adc(sd.points(mix, sd.STREAM_LEARN, 0, LEARN), w.T, w.M, ITERS)
    tasks = [(w.seed, w.n_comp, s, min(CHUNK, w.n_base - s), cb) for s in range(0, w.n_base, CHUNK)]
    saved = {v: os.environ.get(v) for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
    os.environ.update({v: "1" for v in saved})
    try:
        with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
            parts = pool.map(_encode_chunk, tasks)
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    cells = np.concatenate([p[0] for p in parts])
    codes = np.concatenate([p[1] for p in parts])
    index = O.OracleIndex(cb=cb, lists=O.build_lists(cells, codes, np.arange(w.n_base), w.T), variant="global",
                          tables=O.fbpq_tables(cb))
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    for s in range(0, w.n_base, 2_000_000):
        ix.add(sdev.points_cuda(mix, sd.STREAM_BASE, s, min(2_000_000, w.n_base - s)))
    ix.finalize()
    q = sdev.points_cuda(mix, sd.STREAM_QUERY, 0, w.n_query)
    torch.cuda.synchronize()
    return dict(w=w, mix=mix, index=index, ix=ix, q=q, qh=sd.points(mix, sd.STREAM_QUERY, 0, max(SAMPLE) + 1))


def test_full_lists_bit_exact(full):
    a = full["ix"].arrays()
    lists = full["index"].lists
    assert np.array_equal(a["offsets"].cpu().numpy().astype(np.int64), lists.offsets)
    assert np.array_equal(a["codes"].cpu().numpy(), lists.codes)
    assert np.array_equal(a["ids"].cpu().numpy().astype(np.int64), lists.ids)


@pytest.mark.parametrize("L", [1_000, 10_000, 100_000])
def test_full_search_sampled(full, L):
    from oracle import bpq_oracle as O
    k = 100
    ids, dists = full["ix"].search(full["q"], L, k, "fbpq")
    full["ix"].search_status()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    exact = 0
    for n in SAMPLE:
        o_ids, o_d, _, _ = O.search_one(full["index"], full["qh"][n], L, k, "fbpq", traversal="full_sort")
        exact += assert_topk_match(ids[n:n + 1], dists[n:n + 1], o_ids[None], o_d[None])
    assert exact == len(SAMPLE)  # integer data: FP32 sums are exact


@pytest.mark.parametrize("L", [10_000, 100_000])
def test_full_traversal_sampled(full, L):
    """The visit order (the warp pass and the CTA fallback pass) equals the full sort of
    the T^2 cells restricted to non-empty cells, on sampled queries."""
    from oracle import bpq_oracle as O
    from tests.parity import cells_from_gpu
    index = full["index"]
    counts = index.lists.counts()
    cap = int(min(L, (counts > 0).sum()))
    cells, ncells, npoints = full["ix"].traverse(full["q"], L, cap)
    got = cells_from_gpu(cells.cpu().numpy(), ncells.cpu().numpy())
    npoints = npoints.cpu().numpy()
    for n in SAMPLE:
        d1, d2 = O.coarse_distances(full["qh"][n], index.cb)
        oc, _, total = O.traverse_full_sort(d1, d2, counts, L)
        assert np.array_equal(got[n][0], oc[counts[oc] > 0]) and npoints[n] == total


def test_full_reconstruction_and_table_scorers_agree(full):
    """The three scorers return the same lists at the benchmark's size (Eq. 8 vs Eq. 9)."""
    a = [t.cpu().numpy() for t in full["ix"].search(full["q"], 10_000, 100, "fbpq")]
    for scorer in ("fbpq_tables", "recon"):
        b = [t.cpu().numpy() for t in full["ix"].search(full["q"], 10_000, 100, scorer)]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_full_batch_equals_small_batches(full):
    """Queries are independent (each CTA or warp owns one query): a batch of 10k gives the
    same lists as five batches of 2000."""
    import torch
    a = [t.cpu().numpy() for t in full["ix"].search(full["q"], 10_000, 100, "fbpq")]
    parts = [full["ix"].search(full["q"][i:i + 2000], 10_000, 100, "fbpq") for i in range(0, full["q"].shape[0], 2000)]
    b = [torch.cat([p[j] for p in parts]).cpu().numpy() for j in range(2)]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("L", [10_000, 100_000])
def test_full_overlapped_passes_equal_separate_calls(full, L):
    """bpq_search scans the queries the traversal's warp pass finished while, on a second
    stream, the CTA pass takes the queries handed over to it (about 7 % at L = 10k, all at
    L = 100k) and then scans them; every query's list equals the one of the separate
    traversal and scan calls, which run one pass after the other."""
    ix, q = full["ix"], full["q"][:4000]
    ids, dists = ix.search(q, L, 100, "fbpq")
    ix.search_status()
    cap = int(min(L, ix.info().n_nonempty))
    _, _, lut = ix.query_tables(q)
    cells, ncells, _ = ix.traverse(q, L, cap)
    ids2, dists2 = ix.scan(q, lut, cells, ncells, 100, "fbpq")
    assert np.array_equal(ids.cpu().numpy(), ids2.cpu().numpy())
    assert np.array_equal(dists.cpu().numpy(), dists2.cpu().numpy())


def test_full_traversal_all_queries(full):
    """Every query of the 10k batch, not a sample: the warp pass (with its grid rebuilds) and
    the CTA pass emit exactly the multi-sequence order's non-empty cells and L' (§2.3.3)."""
    import synthdata as sd
    from oracle import bpq_oracle as O
    from tests.parity import cells_from_gpu
    index = full["index"]
    counts = index.lists.counts()
    L = 10_000
    cap = int(min(L, (counts > 0).sum()))
    cells, ncells, npoints = full["ix"].traverse(full["q"], L, cap)
    got = cells_from_gpu(cells.cpu().numpy(), ncells.cpu().numpy())
    npoints = npoints.cpu().numpy()
    qh = sd.points(full["mix"], sd.STREAM_QUERY, 0, full["w"].n_query)
    for n in range(len(qh)):
        d1, d2 = O.coarse_distances(qh[n], index.cb)
        oc, _, total = O.traverse_multisequence(d1, d2, counts, L)
        assert np.array_equal(got[n][0], oc[counts[oc] > 0]) and npoints[n] == total, n


def test_full_search_all_queries(full):
    """Every query of the 10k batch at L = 10k (the benchmark's launch): the GPU's top-100 ids
    and distances equal the oracle's (multi-sequence traversal, FP64 FBPQ distances), so
    recall@1/10/100 against any ground truth is identical too."""
    import synthdata as sd
    from oracle import bpq_oracle as O
    L, k = 10_000, 100
    ids, dists = full["ix"].search(full["q"], L, k, "fbpq")
    full["ix"].search_status()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    qh = sd.points(full["mix"], sd.STREAM_QUERY, 0, full["w"].n_query)
    exact = 0
    for n in range(len(qh)):
        o_ids, o_d, _, _ = O.search_one(full["index"], qh[n], L, k, "fbpq")
        exact += assert_topk_match(ids[n:n + 1], dists[n:n + 1], o_ids[None], o_d[None])
    assert exact == len(qh)
