"""Layouts of the search over several GPUs (one process per GPU).

* Replicas: every rank holds the whole index and answers its own batch of
  queries; the only collective is the timing reduction (max over ranks).
* Point shards: rank r holds the points with ids in its range.  Every shard
  traverses the same cells (the traversal's stopping rule uses the per-cell
  counts of the whole index, so the visited cells and L' are those of one index),
  scores the candidates it holds and keeps its k best; one gather and a merge by
  (distance, id) then give exactly the single-index answer, because the k best
  of a union are among the union of the parts' k best.

Queries are independent (§2.3.3), so neither layout has another exchange step.
"""
from __future__ import annotations

import numpy as np


def replica_queries(rank: int, nq_per_rank: int) -> tuple[int, int]:
    """(start, count) of the query batch of one replica rank."""
    return rank * nq_per_rank, nq_per_rank


def shard_points(n: int, rank: int, world: int) -> tuple[int, int]:
    """(start, count) of the contiguous id range of one point shard (sizes differ by at most 1)."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def merge_topk(ids, dists, k: int):
    """Merge per-shard lists ids, dists of shape (S, nq, k_s) into the k best per
    query by (distance, id), ascending; id -1 / +inf entries are padding and sort
    last.  Returns (ids (nq, k) int64, dists (nq, k) float64)."""
    ids = np.asarray(ids, dtype=np.int64)
    dists = np.asarray(dists, dtype=np.float64)
    S, nq, ks = ids.shape
    ids = ids.transpose(1, 0, 2).reshape(nq, S * ks)
    dists = dists.transpose(1, 0, 2).reshape(nq, S * ks)
    pad = ids < 0
    key_id = np.where(pad, np.iinfo(np.int64).max, ids)
    out_i = np.full((nq, k), -1, dtype=np.int64)
    out_d = np.full((nq, k), np.inf)
    for n in range(nq):
        order = np.lexsort((key_id[n], dists[n]))[:k]
        keep = order[~pad[n, order]]
        out_i[n, :len(keep)] = ids[n, keep]
        out_d[n, :len(keep)] = dists[n, keep]
    return out_i, out_d


def global_cell_counts(local_counts, device=None, group=None):
    """The whole index's per-cell counts: the sum over the point shards of each rank's
    counts (numpy int64, T*T), by one all-reduce; every rank gets the same array."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(local_counts, dtype=np.int64), device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def gather_merge(ids, dists, k: int, group=None):
    """All-gather every rank's (nq, k) lists (torch tensors on the backend's device)
    and merge them on every rank.  Returns numpy (ids, dists)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(world)]
    gd = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(gi, ids, group=group)
    dist.all_gather(gd, dists, group=group)
    return merge_topk(np.stack([t.cpu().numpy() for t in gi]), np.stack([t.cpu().numpy() for t in gd]), k)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest value over all ranks (the timing rule of a multi-GPU step)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
