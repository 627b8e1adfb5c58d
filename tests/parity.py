"""Comparison helpers for GPU-vs-oracle parity tests."""
import numpy as np

# Distance tolerance: 1e-4 relative, with a floor for values near zero where the
# FBPQ sum cancels (|d_gpu - d_oracle| <= 1e-4 * max(|d_oracle|, 1)).
RTOL = 1e-4


def close(gpu, ora, rtol=RTOL):
    gpu = np.asarray(gpu, np.float64)
    ora = np.asarray(ora, np.float64)
    both_inf = np.isinf(gpu) & np.isinf(ora)
    tol = rtol * np.maximum(np.abs(np.where(np.isinf(ora), 0, ora)), 1.0)
    diff = np.where(both_inf, 0.0, gpu) - np.where(both_inf, 0.0, ora)
    return both_inf | (np.abs(diff) <= tol)


def assert_topk_match(g_ids, g_d, o_ids, o_d, rtol=RTOL):
    """Top-k lists agree: distances rank by rank within tolerance; ids equal except
    inside groups of near-equal distances, where the id sets must agree; entries at
    the k-th boundary that tie within tolerance are allowed to differ.  Returns the
    number of queries whose lists are bit-identical."""
    g_ids, o_ids = np.asarray(g_ids), np.asarray(o_ids)
    assert g_ids.shape == o_ids.shape
    ok = close(g_d, o_d, rtol)
    assert ok.all(), f"distances differ at {np.argwhere(~ok)[:5].tolist()}"
    exact = 0
    for n in range(len(g_ids)):
        if np.array_equal(g_ids[n], o_ids[n]):
            exact += 1
            continue
        kth = o_d[n][-1]
        near_kth = close(o_d[n], np.full_like(o_d[n], kth), rtol)
        firm = ~near_kth
        assert set(g_ids[n][firm].tolist()) == set(o_ids[n][firm].tolist()), f"query {n}: ids differ"
    return exact


def cells_from_gpu(cells, ncells):
    """Unpack bpq_cell records (int32 (nq, cap, 4)) into per-query lists of (cell, begin, count, key)."""
    cells = np.asarray(cells)
    out = []
    for n, c in enumerate(np.asarray(ncells)):
        rec = cells[n, :c]
        out.append((rec[:, 0].view(np.uint32).astype(np.int64), rec[:, 1].view(np.uint32).astype(np.int64),
                    rec[:, 2].view(np.uint32).astype(np.int64), rec[:, 3].view(np.float32).astype(np.float64)))
    return out
