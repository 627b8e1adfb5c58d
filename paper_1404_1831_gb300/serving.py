"""Online serving of a query stream: Poisson arrivals, batching.

Two request loops over the same resident index, both measured from a query's
arrival to the moment its results are in host memory; each query keeps its own
candidate budget L.

* ``Server`` / ``serve_continuous``: continuous batching in libbpq
  (``bpq_server_*``): a pool of slots, each one batch in flight on its own CUDA
  stream with its own device workspace and page-locked buffers; arrived requests
  are admitted into free slots while earlier batches are still on the GPU, so
  batches overlap on the device, and a batch takes only as many requests as its
  workspace holds at their budgets (admission by device memory), optionally one
  budget class at a time.
* ``serve``: the baseline queue -- whenever the server is free it takes every
  arrived query (at most ``max_batch``) and answers them with one blocking
  ``bpq_search_host`` call.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time

import numpy as np

from . import SCORERS, ServerConfig, ServerStats, _check, _stream, lib


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


class Server:
    """Continuous-batching server over a finalized index (bpq_server_* of libbpq)."""

    def __init__(self, index, k=100, scorer="fbpq", slots=3, max_batch=4096, L_max=100_000,
                 device_bytes=6 << 30, group_by_budget=True):
        self.index, self.k = index, k
        self.D = index.params.D
        cfg = ServerConfig(slots=slots, k=k, scorer=SCORERS[scorer], group_by_budget=1 if group_by_budget else 0,
                           max_batch=max_batch, L_max=L_max, device_bytes=device_bytes)
        h = ctypes.c_void_p()
        _check(lib().bpq_server_create(ctypes.byref(h), index._h, ctypes.byref(cfg)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().bpq_server_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def submit(self, queries, L):
        """Queues requests; returns the first request number."""
        q = np.ascontiguousarray(queries, dtype=np.float32).reshape(-1, self.D)
        Ls = np.ascontiguousarray(np.broadcast_to(np.asarray(L, dtype=np.int64), (q.shape[0],)))
        first = ctypes.c_int64()
        _check(lib().bpq_server_submit(self._h, q.ctypes.data, Ls.ctypes.data, q.shape[0], ctypes.byref(first)))
        return first.value

    def progress(self, wait=False):
        _check(lib().bpq_server_progress(self._h, 1 if wait else 0))

    def take(self, max_n=4096):
        """Finished requests: (request numbers, ids (n, k), dists (n, k), latency seconds)."""
        req = np.empty(max_n, dtype=np.int64)
        ids = np.empty((max_n, self.k), dtype=np.int32)
        dists = np.empty((max_n, self.k), dtype=np.float32)
        lat = np.empty(max_n, dtype=np.float64)
        n = ctypes.c_int64()
        _check(lib().bpq_server_take(self._h, max_n, req.ctypes.data, ids.ctypes.data, dists.ctypes.data,
                                     lat.ctypes.data, ctypes.byref(n)))
        m = n.value
        return req[:m], ids[:m], dists[:m], lat[:m]

    def stats(self):
        st = ServerStats()
        _check(lib().bpq_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def run_trace(self, queries, L, arrivals):
        """Serves a recorded trace (arrival seconds, non-decreasing); returns a ServeResult."""
        q = np.ascontiguousarray(queries, dtype=np.float32)
        Ls = np.ascontiguousarray(L, dtype=np.int64)
        arr = np.ascontiguousarray(arrivals, dtype=np.float64)
        n = len(arr)
        ids = np.empty((n, self.k), dtype=np.int32)
        dists = np.empty((n, self.k), dtype=np.float32)
        lat = np.empty(n, dtype=np.float64)
        b0 = self.stats()["batches"]
        t0 = time.perf_counter()
        _check(lib().bpq_server_run_trace(self._h, q.ctypes.data, Ls.ctypes.data, arr.ctypes.data, n,
                                          ids.ctypes.data, dists.ctypes.data, lat.ctypes.data))
        wall = time.perf_counter() - t0
        nb = self.stats()["batches"] - b0
        return ServeResult(latency_s=lat, batch_sizes=np.full(max(nb, 1), n / max(nb, 1)),
                           wall_s=max(wall - float(arr[0]), 1e-9), ids=ids, dists=dists)


def serve_continuous(index, queries, L, arrivals, k=100, scorer="fbpq", slots=3, max_batch=4096,
                     L_max=None, device_bytes=6 << 30, group_by_budget=True) -> ServeResult:
    """Continuous batching of a Poisson (or any recorded) arrival trace."""
    L = np.asarray(L, dtype=np.int64)
    srv = Server(index, k=k, scorer=scorer, slots=slots, max_batch=max_batch,
                 L_max=int(L.max()) if L_max is None else L_max, device_bytes=device_bytes,
                 group_by_budget=group_by_budget)
    try:
        res = srv.run_trace(queries, L, arrivals)
        res.stats = srv.stats()
    finally:
        srv.close()
    return res
