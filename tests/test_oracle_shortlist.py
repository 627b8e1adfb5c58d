"""Pins of the oracle's int8-table shortlist search (a precision variant of §3.1)."""
import numpy as np
import pytest

from oracle import bpq_oracle as O


@pytest.fixture(scope="module")
def small():
    import synthdata as sd
    w = sd.TINY
    mix = sd.make_mixture(w.seed, w.n_comp, w.dim)
    cb = O.train_multi_d_adc(sd.points(mix, sd.STREAM_LEARN, 0, w.n_learn), w.T, w.M, 3)
    index = O.build_index(cb, sd.points(mix, sd.STREAM_BASE, 0, 20_000))
    return dict(cb=cb, index=index, q=sd.points(mix, sd.STREAM_QUERY, 0, 6))


def test_table_and_cross_terms_reproduce_eq8(small):
    """key(i,j) + sum_k lut[k][c_k] + cross(p) is the FBPQ distance of Eqs. 8-9,
    which dist_fbpq expands term by term (and which is pinned to the explicit
    reconstruction elsewhere): equal exactly on integer data."""
    cb, index = small["cb"], small["index"]
    lists = index.lists
    rng = np.random.default_rng(1)
    pos = rng.integers(0, len(lists.ids), 500)
    cell = np.searchsorted(lists.offsets, pos, side="right") - 1
    codes = lists.codes[pos].astype(np.int64)
    for q in small["q"][:3]:
        d1, d2 = O.coarse_distances(q, cb)
        lut = O.pq_table(q, cb)
        got = (d1[cell // cb.T] + d2[cell % cb.T] + lut[np.arange(cb.M)[None, :], codes].sum(1)
               + O.point_cross(cb, index.tables, cell, codes))
        assert np.array_equal(got, O.dist_fbpq(q, cb, index.tables, cell, codes))


def test_quantized_table_bounds(small):
    for q in small["q"]:
        lut = O.pq_table(q, small["cb"])
        q8, s = O.quantize_table_int8(lut)
        lo = lut.min(1)
        assert q8.dtype == np.int64 and q8.min() >= 0 and q8.max() <= 255
        assert np.all(q8.min(1) == 0)                    # every table's minimum maps to 0
        widest = np.argmax(lut.max(1) - lo)
        assert q8[widest].max() == 255                    # the widest table spans the full range
        err = np.abs(lo[:, None] + np.float64(s) * q8 - lut)
        assert err.max() <= 0.5 * s * (1 + 1e-5)         # round to nearest: half a step
    q8, s = O.quantize_table_int8(np.full((4, 256), 7.0))
    assert s == 1 and not q8.any()


def test_score_is_distance_within_quantization_bound(small):
    """score = exact distance - sum_k lo_k up to M * s / 2 (plus FP32 rounding)."""
    cb, index = small["cb"], small["index"]
    lists = index.lists
    q = small["q"][0]
    d1, d2 = O.coarse_distances(q, cb)
    cells, _, _ = O.traverse_full_sort(d1, d2, lists.counts(), 3000)
    pos = O.candidates(cells, lists)
    cell = np.repeat(cells, lists.counts()[cells])
    codes = lists.codes[pos].astype(np.int64)
    lut = O.pq_table(q, cb)
    q8, s = O.quantize_table_int8(lut)
    key32 = (d1[cell // cb.T] + d2[cell % cb.T]).astype(np.float32)
    cross32 = O.point_cross(cb, index.tables, cell, codes).astype(np.float32)
    score = ((key32 + cross32) + s * q8[np.arange(cb.M)[None, :], codes].sum(1).astype(np.float32))
    exact = O.dist_fbpq(q, cb, index.tables, cell, codes)
    dev = np.abs(score.astype(np.float64) - (exact - lut.min(1).sum()))
    assert dev.max() <= cb.M * 0.5 * s + 1e-6 * np.abs(exact).max() + 1.0


def test_full_shortlist_equals_fbpq_search(small):
    for q in small["q"]:
        a = O.search_one(small["index"], q, 3000, 50, "fbpq", traversal="full_sort")
        b = O.search_shortlist_one(small["index"], q, 3000, 50, 10 ** 6)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_short_shortlist_keeps_distances_exact(small):
    """Whatever the shortlist keeps is re-scored exactly: every returned distance
    is the FBPQ distance of the returned id, and the list is a subset ranked like
    the full search."""
    index = small["index"]
    for q in small["q"]:
        ids, d = O.search_shortlist_one(index, q, 3000, 50, 100)
        full_ids, full_d, _, _ = O.search_one(index, q, 3000, 10 ** 4, "fbpq", traversal="full_sort")
        where = {int(i): float(v) for i, v in zip(full_ids, full_d)}
        assert all(where[int(i)] == float(v) for i, v in zip(ids, d) if i >= 0)
        assert np.all(np.diff(d) >= 0)


def test_fp16_table_is_nearest_value_at_smallest_power_of_two_step(small):
    """Every stored entry is the FP16 value nearest to (lut - lo_k) / s: neither FP16
    neighbour is closer (checked through np.nextafter, not the conversion); s is the
    smallest power of two >= 1 that keeps the widest table finite."""
    for q in small["q"][:3]:
        lut = O.pq_table(q, small["cb"])
        h, s = O.quantize_table_fp16(lut)
        assert h.dtype == np.float16 and np.isfinite(h).all()
        x = (lut - lut.min(1)[:, None]) / float(s)
        assert x.max() <= 65504.0 and (s == 1 or x.max() * 2 > 65504.0)
        assert float(s) == 2.0 ** round(np.log2(float(s)))
        hv = h.astype(np.float64)
        up = np.nextafter(h, np.float16(np.inf)).astype(np.float64)
        dn = np.nextafter(h, np.float16(-np.inf)).astype(np.float64)
        err = np.abs(hv - x)
        assert np.all(err <= np.abs(up - x)) and np.all(err <= np.abs(dn - x))


def test_fp16_small_integer_tables_are_exact():
    """Integers up to 2048 are FP16 values: such a table is stored exactly (s = 1)."""
    rng = np.random.default_rng(3)
    lut = rng.integers(-1000, 1048, size=(8, 256)).astype(np.float64)
    h, s = O.quantize_table_fp16(lut)
    assert s == 1
    assert np.array_equal(lut.min(1)[:, None] + h.astype(np.float64), lut)


def test_fp16_score_is_distance_within_rounding_bound(small):
    cb, index = small["cb"], small["index"]
    lists = index.lists
    q = small["q"][1]
    d1, d2 = O.coarse_distances(q, cb)
    cells, _, _ = O.traverse_full_sort(d1, d2, lists.counts(), 3000)
    pos = O.candidates(cells, lists)
    cell = np.repeat(cells, lists.counts()[cells])
    codes = lists.codes[pos].astype(np.int64)
    lut = O.pq_table(q, cb)
    h, s = O.quantize_table_fp16(lut)
    key32 = (d1[cell // cb.T] + d2[cell % cb.T]).astype(np.float32)
    cross32 = O.point_cross(cb, index.tables, cell, codes).astype(np.float32)
    score = (key32 + cross32) + O.shortlist_part(q, cb, codes, "fp16")
    exact = O.dist_fbpq(q, cb, index.tables, cell, codes)
    x = lut - lut.min(1)[:, None]
    tab_err = float(s) * (2.0 ** -11) * x[np.arange(cb.M)[None, :], codes].sum(1)
    dev = np.abs(score.astype(np.float64) - (exact - lut.min(1).sum()))
    assert np.all(dev <= tab_err + cb.M * float(s) * 65504.0 * 2.0 ** -23 + 1e-6 * np.abs(exact).max() + 1.0)


def test_fp16_full_shortlist_equals_fbpq_search(small):
    for q in small["q"][:3]:
        a = O.search_one(small["index"], q, 3000, 50, "fbpq", traversal="full_sort")
        b = O.search_shortlist_one(small["index"], q, 3000, 50, 10 ** 6, "fp16")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
