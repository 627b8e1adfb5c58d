"""GPU parity on the tiny workload (100k SIFT-shaped points, T = 64, M = 8): every
step of the CUDA path through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match, cells_from_gpu, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def gpu(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    w = t["w"]
    learn = torch.as_tensor(t["learn"], dtype=torch.float32, device=DEV)
    ix = bpq.Index.train(learn, w.T, w.M, iters=w.kmeans_iters)
    base = torch.as_tensor(t["base"], dtype=torch.float32, device=DEV)
    ix.add(base)
    ix.finalize()
    q = torch.as_tensor(t["queries"], dtype=torch.float32, device=DEV)
    return dict(ix=ix, q=q, base=base)


def test_device_generator_matches_numpy(tiny_oracle):
    import synthdata as sd
    from synthdata import device as sdev
    mix = tiny_oracle["mix"]
    for stream, start, count in ((sd.STREAM_BASE, 0, 4000), (sd.STREAM_QUERY, 0, 100), (sd.STREAM_BASE, 99_000, 1000)):
        a = sdev.points_cuda(mix, stream, start, count).cpu().numpy()
        assert np.array_equal(a, sd.points(mix, stream, start, count).astype(np.float32))


def test_training_is_bit_exact(gpu, tiny_oracle):
    cb = tiny_oracle["cb"]
    a = gpu["ix"].arrays()
    assert np.array_equal(a["C1"].cpu().numpy(), cb.C1.astype(np.float32))
    assert np.array_equal(a["C2"].cpu().numpy(), cb.C2.astype(np.float32))
    assert np.array_equal(a["R"].cpu().numpy(), cb.R.astype(np.float32))


def test_encode_and_lists_bit_exact(gpu, tiny_oracle):
    cb, lists = tiny_oracle["cb"], tiny_oracle["index"].lists
    cells, codes = gpu["ix"].encode(gpu["base"])
    oc, ok = O.encode_multi_d_adc(tiny_oracle["base"], cb)
    assert np.array_equal(cells.cpu().numpy(), oc) and np.array_equal(codes.cpu().numpy(), ok)
    a = gpu["ix"].arrays()
    assert np.array_equal(a["offsets"].cpu().numpy().astype(np.int64), lists.offsets)
    assert np.array_equal(a["codes"].cpu().numpy(), lists.codes)
    assert np.array_equal(a["ids"].cpu().numpy(), lists.ids)
    info = gpu["ix"].info()
    assert info.n_points == len(lists.ids) and info.n_nonempty == int((lists.counts() > 0).sum())


def test_fbpq_tables_bit_exact(gpu, tiny_oracle):
    tab = tiny_oracle["index"].tables
    a = gpu["ix"].arrays()
    assert np.array_equal(a["X1"].cpu().numpy(), (2 * tab.X1).astype(np.float32))
    assert np.array_equal(a["X2"].cpu().numpy(), (2 * tab.X2).astype(np.float32))


def test_point_cross_terms_bit_exact(gpu, tiny_oracle):
    """The per-point Eq. 9 cross term 2<[c^1_i; c^2_j], r> used by the FBPQ scan."""
    idx = tiny_oracle["index"]
    cb, lists, tab = idx.cb, idx.lists, idx.tables
    cell = np.repeat(np.arange(cb.T * cb.T), lists.counts())
    i, j = cell // cb.T, cell % cb.T
    m2 = cb.M // 2
    codes = lists.codes.astype(np.int64)
    ref = sum(tab.X1[i, k, codes[:, k]] for k in range(m2)) + sum(tab.X2[j, k, codes[:, m2 + k]] for k in range(m2))
    got = gpu["ix"].arrays()["cross"].cpu().numpy()
    assert np.array_equal(got, (2 * ref).astype(np.float32))
    # and it is the explicit 2<c_ij, r> of the reconstruction (Eq. 7)
    xr = O.reconstruct(cb, cell[:5000], lists.codes[:5000])
    cen = np.concatenate([cb.C1[i[:5000]], cb.C2[j[:5000]]], axis=1)
    assert np.array_equal(got[:5000].astype(np.float64), 2 * ((xr - cen) * cen).sum(1))


def test_query_tables_bit_exact(gpu, tiny_oracle):
    cb = tiny_oracle["cb"]
    d1, d2, lut = gpu["ix"].query_tables(gpu["q"])
    d1, d2, lut = d1.cpu().numpy(), d2.cpu().numpy(), lut.cpu().numpy()
    s = cb.sub
    for n, q in enumerate(tiny_oracle["queries"][:20]):
        o1, o2 = O.coarse_distances(q, cb)
        assert np.array_equal(d1[n], o1) and np.array_equal(d2[n], o2)
        ref = np.stack([(cb.R[k] ** 2).sum(1) - 2.0 * (cb.R[k] @ q[k * s:(k + 1) * s].astype(np.float64))
                        for k in range(cb.M)])
        assert np.array_equal(lut[n], ref)


def test_query_tables_all_query_counts(gpu, tiny_oracle):
    """Tile edges of the tensor-core table kernel (128 queries per tile): 1, 127,
    129 and 100 queries give the same rows as the full batch."""
    full = [t.cpu().numpy() for t in gpu["ix"].query_tables(gpu["q"])]
    q = torch.cat([gpu["q"], gpu["q"], gpu["q"]])[:300]
    for n in (1, 127, 129, 300):
        part = [t.cpu().numpy() for t in gpu["ix"].query_tables(q[:n].contiguous())]
        for a, b in zip(full, part):
            m = min(n, 100)
            assert np.array_equal(a[:m], b[:m])


def test_query_tables_fp32_path_for_non_bf16_inputs(gpu, tiny_oracle):
    """Queries (or codebooks) that BF16 cannot hold exactly are tabulated in FP32
    on the CUDA cores: within FP32 rounding of the FP64 definition."""
    import paper_1404_1831_gb300 as bpq
    cb = tiny_oracle["cb"]
    s = cb.sub
    qh = tiny_oracle["queries"][:12].astype(np.float64) + 0.25
    d1, d2, lut = [t.cpu().numpy().astype(np.float64) for t in
                   gpu["ix"].query_tables(torch.as_tensor(qh, dtype=torch.float32, device=DEV))]
    for n, q in enumerate(qh):
        o1, o2 = O.coarse_distances(q, cb)
        assert np.allclose(d1[n], o1, rtol=1e-6, atol=1e-2) and np.allclose(d2[n], o2, rtol=1e-6, atol=1e-2)
        ref = np.stack([(cb.R[k] ** 2).sum(1) - 2.0 * (cb.R[k] @ q[k * s:(k + 1) * s]) for k in range(cb.M)])
        assert np.allclose(lut[n], ref, rtol=1e-6, atol=1e-1)
    C1 = cb.C1.astype(np.float64) + 0.5  # not BF16-exact at these magnitudes
    ix = bpq.Index.create(C1, cb.C2, cb.R)
    d1, _, _ = [t.cpu().numpy().astype(np.float64) for t in ix.query_tables(gpu["q"][:8])]
    for n in range(8):
        q = tiny_oracle["queries"][n].astype(np.float64)
        ref = ((q[None, :cb.D // 2] - C1) ** 2).sum(1)
        assert np.allclose(d1[n], ref, rtol=1e-6, atol=1e-2)


@pytest.mark.parametrize("L", [1, 37, 1000, 10_000, 60_000, 250_000])
def test_traversal_bit_exact(gpu, tiny_oracle, L):
    cb, lists = tiny_oracle["cb"], tiny_oracle["index"].lists
    cap = 4096
    cells, ncells, npoints = gpu["ix"].traverse(gpu["q"], L, cap)
    got = cells_from_gpu(cells.cpu().numpy(), ncells.cpu().numpy())
    npoints = npoints.cpu().numpy()
    counts = lists.counts()
    for n, q in enumerate(tiny_oracle["queries"][:40]):
        d1, d2 = O.coarse_distances(q, cb)
        oc, okeys, total = O.traverse_multisequence(d1, d2, counts, L)
        keep = counts[oc] > 0
        c, b, cnt, key = got[n]
        assert np.array_equal(c, oc[keep]), f"query {n}: cell order differs"
        assert np.array_equal(key, okeys[keep])
        assert np.array_equal(b, lists.offsets[c]) and np.array_equal(cnt, counts[c])
        assert npoints[n] == total


def test_traversal_uneven_budgets(gpu, tiny_oracle):
    cb, lists = tiny_oracle["cb"], tiny_oracle["index"].lists
    rng = np.random.default_rng(7)
    Ls = np.round(10 ** rng.uniform(0, 5, size=len(tiny_oracle["queries"]))).astype(np.int64)
    cells, ncells, npoints = gpu["ix"].traverse(gpu["q"], Ls, 4096)
    got = cells_from_gpu(cells.cpu().numpy(), ncells.cpu().numpy())
    for n, q in enumerate(tiny_oracle["queries"]):
        d1, d2 = O.coarse_distances(q, cb)
        oc, _, total = O.traverse_full_sort(d1, d2, lists.counts(), int(Ls[n]))
        assert np.array_equal(got[n][0], oc[lists.counts()[oc] > 0]) and npoints.cpu().numpy()[n] == total


@pytest.mark.parametrize("scorer", ["fbpq", "fbpq_tables", "recon"])
def test_search_matches_oracle(gpu, tiny_oracle, scorer):
    w = tiny_oracle["w"]
    ids, dists = gpu["ix"].search(gpu["q"], w.L[0], w.k, scorer)
    gpu["ix"].search_status()
    o_ids, o_d, _ = O.search(tiny_oracle["index"], tiny_oracle["queries"], w.L[0], w.k, "fbpq")
    exact = assert_topk_match(ids.cpu().numpy(), dists.cpu().numpy(), o_ids, o_d)
    assert exact == len(o_ids)  # integer data: FP32 sums are exact here
    nn = O.exact_nn(tiny_oracle["base"], tiny_oracle["queries"][:30])
    for R in (1, 10, 100):
        assert O.recall_at(ids.cpu().numpy()[:30], nn, R) == O.recall_at(o_ids[:30], nn, R)


def test_fbpq_equals_reconstruction_on_gpu(gpu):
    a = [t.cpu().numpy() for t in gpu["ix"].search(gpu["q"], 20_000, 100, "fbpq")]
    for other in ("fbpq_tables", "recon"):
        b = [t.cpu().numpy() for t in gpu["ix"].search(gpu["q"], 20_000, 100, other)]
        assert np.array_equal(a[0], b[0]) and close(a[1], b[1]).all()


@pytest.mark.parametrize("k", [1, 7, 128, 129, 300, 1024])
def test_search_k_values(gpu, tiny_oracle, k):
    L = 3000
    ids, dists = gpu["ix"].search(gpu["q"][:12], L, k, "fbpq")
    o_ids, o_d, _ = O.search(tiny_oracle["index"], tiny_oracle["queries"][:12], L, k, "fbpq")
    assert_topk_match(ids.cpu().numpy(), dists.cpu().numpy(), o_ids, o_d)


def test_padding_when_fewer_candidates_than_k(gpu, tiny_oracle):
    ids, dists = gpu["ix"].search(gpu["q"][:10], 1, 1024, "fbpq")
    o_ids, o_d, totals = O.search(tiny_oracle["index"], tiny_oracle["queries"][:10], 1, 1024, "fbpq")
    assert (totals < 1024).any()
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    assert np.array_equal(ids, o_ids)
    assert np.array_equal(np.isinf(dists), np.isinf(o_d))


def test_budget_beyond_index_visits_everything(gpu, tiny_oracle):
    n = len(tiny_oracle["base"])
    _, ncells, npoints = gpu["ix"].traverse(gpu["q"][:4], n + 1000, 4096)
    assert (npoints.cpu().numpy() == n).all()
    assert (ncells.cpu().numpy() == int((tiny_oracle["index"].lists.counts() > 0).sum())).all()


def test_small_workspace_chunks_queries(gpu, tiny_oracle):
    ix = gpu["ix"]
    full = [t.cpu().numpy() for t in ix.search(gpu["q"], 5000, 50)]
    import paper_1404_1831_gb300 as bpq
    one = bpq.lib().bpq_search_workspace_size(ix._h, 1, 5000, 50, 0)
    ws = torch.empty(one * 3, dtype=torch.uint8, device=DEV)
    part = [t.cpu().numpy() for t in ix.search(gpu["q"], 5000, 50, workspace=ws)]
    assert np.array_equal(full[0], part[0]) and np.array_equal(full[1], part[1])
    with pytest.raises(bpq.BpqError):
        ix.search(gpu["q"], 5000, 50, workspace=torch.empty(64, dtype=torch.uint8, device=DEV))


def test_host_buffer_search_equals_device_search(gpu, tiny_oracle):
    a = [t.cpu().numpy() for t in gpu["ix"].search(gpu["q"], 10_000, 100)]
    b = gpu["ix"].search_host(tiny_oracle["queries"].astype(np.float32), 10_000, 100)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_invalid_arguments_are_rejected(gpu):
    import paper_1404_1831_gb300 as bpq
    ix, q = gpu["ix"], gpu["q"][:2]
    for kwargs in (dict(L=0, k=10), dict(L=10, k=0), dict(L=10, k=1025), dict(L=[5, 5, 5], k=3)):
        with pytest.raises((bpq.BpqError, ValueError)):
            ix.search(q, kwargs["L"], kwargs["k"])
    with pytest.raises(bpq.BpqError):
        ix.search(q, 10, 10, "hbpq")  # global codebooks: no local scorer


def test_empty_query_batch_and_empty_index(gpu, tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    ids, dists = gpu["ix"].search(gpu["q"][:0], 100, 10)
    assert ids.shape == (0, 10)
    cb = tiny_oracle["cb"]
    empty = bpq.Index.create(cb.C1, cb.C2, cb.R)
    ids, dists = empty.search(gpu["q"][:3], 100, 5)
    assert (ids.cpu().numpy() == -1).all() and np.isinf(dists.cpu().numpy()).all()


def test_pending_points_block_search_until_finalize(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    cb = tiny_oracle["cb"]
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    base = torch.as_tensor(tiny_oracle["base"][:5000], dtype=torch.float32, device=DEV)
    ix.add(base[:3000])
    q = torch.as_tensor(tiny_oracle["queries"][:4], dtype=torch.float32, device=DEV)
    with pytest.raises(bpq.BpqError) as e:
        ix.search(q, 100, 5)
    assert e.value.code == -8
    ix.finalize()
    ix.add(base[3000:], ids=torch.arange(3000, 5000, dtype=torch.int32, device=DEV))
    ix.finalize()
    oix = O.build_index(cb, tiny_oracle["base"][:5000])
    got = [t.cpu().numpy() for t in ix.search(q, 500, 20)]
    o_ids, o_d, _ = O.search(oix, tiny_oracle["queries"][:4], 500, 20)
    assert_topk_match(got[0], got[1], o_ids, o_d)
    a = ix.arrays()
    assert np.array_equal(a["ids"].cpu().numpy(), oix.lists.ids)


def test_save_load_roundtrip_and_corruption(gpu, tmp_path):
    import paper_1404_1831_gb300 as bpq
    path = tmp_path / "idx.bpq"
    gpu["ix"].save(path)
    ix2 = bpq.Index.load(path)
    a = [t.cpu().numpy() for t in gpu["ix"].search(gpu["q"], 2000, 30)]
    b = [t.cpu().numpy() for t in ix2.search(gpu["q"], 2000, 30)]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0xFF
    bad = tmp_path / "bad.bpq"
    bad.write_bytes(bytes(raw))
    with pytest.raises(bpq.BpqError) as e:
        bpq.Index.load(bad)
    assert e.value.code == -4


def test_serving_answers_equal_batch_search(gpu, tiny_oracle):
    """The Poisson serving loop (dynamic batches through bpq_search_host) returns the
    same lists as one batch search with the same per-query budgets."""
    from paper_1404_1831_gb300 import serving
    q = tiny_oracle["queries"].astype(np.float32)
    n = len(q)
    L = np.resize(np.array([1_000, 10_000, 3_000], dtype=np.int64), n)
    res = serving.serve(gpu["ix"], q, L, serving.poisson_arrivals(n, 20_000.0, 5), k=50, max_batch=16)
    ids, dists = gpu["ix"].search(gpu["q"], L, 50)
    assert np.array_equal(res.ids, ids.cpu().numpy()) and np.array_equal(res.dists, dists.cpu().numpy())
    assert res.batch_sizes.sum() == n and res.batch_sizes.max() <= 16
    assert (res.latency_s > 0).all()
    s = res.summary()
    assert s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]


@pytest.mark.parametrize("k", [10, 100, 128])
def test_search_with_large_tie_groups(tiny_oracle, k):
    """40 points, each added 500 times under distinct ids: every distance is shared by
    500 candidates, so the scan's buffers fill with entries tied at their cut value
    (the exact re-rank by (distance, id)) and the final survivors exceed 128 (the rank
    count); the lists equal the oracle's, ties by id."""
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    cb = t["cb"]
    base = np.repeat(t["base"][:40], 500, axis=0)
    index = O.build_index(cb, base)
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    ix.add(torch.as_tensor(base, dtype=torch.float32, device=DEV))
    ix.finalize()
    q = t["queries"][:8]
    ids, dists = ix.search(torch.as_tensor(q, dtype=torch.float32, device=DEV), len(base), k, "fbpq")
    o_ids, o_d, _ = O.search(index, q, len(base), k, "fbpq")
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    assert np.array_equal(ids, o_ids)
    assert np.array_equal(dists.astype(np.float64), o_d)
    ix.close()
