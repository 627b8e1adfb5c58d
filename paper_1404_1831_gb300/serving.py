"""Online serving of a query stream: Poisson arrivals, dynamic batching.

Queries arrive at the times of a seeded Poisson process.  Whenever the server is
free it takes every query that has arrived (at most `max_batch`, oldest first)
and answers them with one `bpq_search_host` call: the batch is copied to the
GPU, searched (query tables, traversal, scan, top-k) and the results copied
back to host memory.  A query's latency is the time from its arrival to the
moment its batch's results are in host memory.  Each query keeps its own
candidate budget L.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import SCORERS, _check, _stream, lib


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from the start) of n queries at `rate` queries/s."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


@dataclasses.dataclass
class ServeResult:
    latency_s: np.ndarray   # (n,) arrival -> results in host memory
    batch_sizes: np.ndarray  # queries per search call, in order
    wall_s: float           # first arrival -> last completion
    ids: np.ndarray         # (n, k) int32
    dists: np.ndarray       # (n, k) float32

    def summary(self) -> dict:
        lat_ms = self.latency_s * 1e3
        return {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "mean_ms": float(lat_ms.mean()), "max_ms": float(lat_ms.max()),
                "queries": int(len(lat_ms)), "served_qps": float(len(lat_ms) / self.wall_s),
                "batches": int(len(self.batch_sizes)), "mean_batch": float(self.batch_sizes.mean())}


def serve(index, queries: np.ndarray, L: np.ndarray, arrivals: np.ndarray, k: int = 100, scorer: str = "fbpq",
          max_batch: int = 4096, stream=None) -> ServeResult:
    """Serves queries (n, D) float32 (host) with budgets L (n,) arriving at `arrivals`
    (sorted, seconds).  Returns per-query latencies and the answers."""
    queries = np.ascontiguousarray(queries, dtype=np.float32)
    L = np.ascontiguousarray(L, dtype=np.int64)
    arrivals = np.asarray(arrivals, dtype=np.float64)
    n = len(arrivals)
    assert queries.shape[0] == n and L.shape == (n,)
    ids = np.empty((n, k), dtype=np.int32)
    dists = np.empty((n, k), dtype=np.float32)
    lat = np.empty(n)
    sizes = []
    h, sc, st = index._h, SCORERS[scorer], _stream(stream)
    D = queries.shape[1]
    qb, Lb, ib, db = queries.ctypes.data, L.ctypes.data, ids.ctypes.data, dists.ctypes.data
    i = 0
    t0 = time.perf_counter()
    while i < n:
        now = time.perf_counter() - t0
        while now < arrivals[i]:  # idle until the next arrival
            gap = arrivals[i] - now
            if gap > 3e-4:
                time.sleep(gap - 2e-4)
            now = time.perf_counter() - t0
        j = min(n, i + max_batch, int(np.searchsorted(arrivals, now, side="right")))
        _check(lib().bpq_search_host(h, qb + i * D * 4, j - i, Lb + i * 8, 1, k, sc, ib + i * k * 4,
                                     db + i * k * 4, st))
        done = time.perf_counter() - t0
        lat[i:j] = done - arrivals[i:j]
        sizes.append(j - i)
        i = j
    wall = (time.perf_counter() - t0) - arrivals[0]
    return ServeResult(latency_s=lat, batch_sizes=np.asarray(sizes), wall_s=wall, ids=ids, dists=dists)


def saturated_qps(index, queries: np.ndarray, L: np.ndarray, k: int = 100, scorer: str = "fbpq",
                  batch: int = 4096, batches: int = 8, stream=None) -> float:
    """Queries/s of back-to-back full batches of distinct queries through the same
    host-buffer call (the first batch, which sizes the buffers, is not timed)."""
    queries = np.ascontiguousarray(queries, dtype=np.float32)
    L = np.ascontiguousarray(L, dtype=np.int64)
    n = min(len(queries), batch * (batches + 1))
    ids = np.empty((batch, k), dtype=np.int32)
    dists = np.empty((batch, k), dtype=np.float32)
    sc, st = SCORERS[scorer], _stream(stream)
    D = queries.shape[1]
    done, t = 0, None
    for b0 in range(0, n - batch + 1, batch):
        if b0 == batch:
            t = time.perf_counter()
        _check(lib().bpq_search_host(index._h, queries.ctypes.data + b0 * D * 4, batch, L.ctypes.data + b0 * 8, 1,
                                     k, sc, ids.ctypes.data, dists.ctypes.data, st))
        if b0 >= batch:
            done += batch
    return done / (time.perf_counter() - t)
