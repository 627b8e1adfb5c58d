"""Multi-GPU layouts on CPU ranks (gloo, world size 2): the max-over-ranks timing
reduction, and point sharding — every shard traverses with the whole index's cell
counts, keeps its own k best, and the gathered merge equals the single-index answer."""
import os
import socket

import numpy as np
import pytest

from paper_1404_1831_gb300 import multi

torch = pytest.importorskip("torch")


def test_shard_points_partition():
    for n, world in ((10, 3), (7, 7), (5, 8), (100_000, 4)):
        parts = [multi.shard_points(n, r, world) for r in range(world)]
        assert parts[0][0] == 0 and sum(c for _, c in parts) == n
        assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    assert multi.replica_queries(3, 10_000) == (30_000, 10_000)


def test_merge_topk_equals_sort_of_union():
    rng = np.random.default_rng(0)
    S, nq, k = 3, 20, 7
    d = rng.integers(0, 30, (S, nq, k)).astype(np.float64)  # many ties
    ids = rng.permutation(S * nq * k).reshape(S, nq, k)
    d[1, :3, 4:] = np.inf
    ids[1, :3, 4:] = -1  # padding
    d.sort(axis=2)
    mi, md = multi.merge_topk(ids, d, k)
    for n in range(nq):
        allid = ids[:, n, :].ravel()
        alld = d[:, n, :].ravel()
        real = allid >= 0
        order = np.lexsort((allid[real], alld[real]))[:k]
        assert np.array_equal(mi[n, :len(order)], allid[real][order])
        assert np.array_equal(md[n, :len(order)], alld[real][order])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import synthdata as sd
    from oracle import bpq_oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = multi.max_over_ranks(rank + 1.5)
        mix = sd.make_mixture(7, 32)
        learn = sd.points(mix, sd.STREAM_LEARN, 0, 4000)
        base = sd.points(mix, sd.STREAM_BASE, 0, 12_000)
        queries = sd.points(mix, sd.STREAM_QUERY, 0, 6)
        cb = O.train_multi_d_adc(learn, 16, 8, 3)  # deterministic: the same codebooks on every rank
        full = O.build_index(cb, base)
        start, count = multi.shard_points(len(base), rank, world)
        shard = O.build_index(cb, base[start:start + count], ids=np.arange(start, start + count))
        # the whole index's counts, summed over the shards by one all-reduce
        gcounts = multi.global_cell_counts(shard.lists.counts())
        k = 30
        ids = np.empty((len(queries), k), dtype=np.int64)
        dd = np.empty((len(queries), k))
        for n, q in enumerate(queries):
            ids[n], dd[n], _, _ = O.search_one(shard, q, 2000, k, "fbpq", traversal="full_sort",
                                               cut_counts=gcounts)
        mi, md = multi.gather_merge(torch.as_tensor(ids), torch.as_tensor(dd), k)
        if rank == 0:
            ref_i, ref_d, _ = O.search(full, queries, 2000, k, "fbpq", traversal="full_sort")
            np.savez(os.path.join(out_dir, "r.npz"), mi=mi, md=md, ri=ref_i, rd=ref_d, mx=mx,
                     gc=np.array_equal(gcounts, full.lists.counts()))
    finally:
        dist.destroy_process_group()


def test_sharded_search_merges_to_single_index_answer(tmp_path):
    import torch.multiprocessing as tmp
    tmp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r = np.load(tmp_path / "r.npz")
    assert float(r["mx"]) == 2.5
    assert bool(r["gc"])  # summed shard counts = the single index's counts
    assert np.array_equal(r["mi"], r["ri"]) and np.array_equal(r["md"], r["rd"])
