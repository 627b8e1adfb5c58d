"""Pins for the cell traversal (§2.3.3): the multi-sequence heap against the
plain full-sort definition, plus the invariants of the visit order."""
import numpy as np
import pytest

from oracle import bpq_oracle as O


def random_case(rng, T, ties):
    hi = 6 if ties else 10_000
    d1 = rng.integers(0, hi, size=T).astype(np.float64)
    d2 = rng.integers(0, hi, size=T).astype(np.float64)
    counts = rng.integers(0, 4, size=T * T) * (rng.random(T * T) < 0.6)
    return d1, d2, counts


@pytest.mark.parametrize("seed", range(40))
def test_multisequence_equals_full_sort(seed):
    rng = np.random.default_rng(seed)
    T = int(rng.integers(1, 24))
    d1, d2, counts = random_case(rng, T, ties=seed % 2 == 0)
    total = int(counts.sum())
    for L in (1, 2, 5, max(1, total // 3), max(1, total), total + 5):
        a = O.traverse_full_sort(d1, d2, counts, L)
        b = O.traverse_multisequence(d1, d2, counts, L)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_full_sort_against_hand_enumeration():
    d1 = np.array([3.0, 1.0, 2.0])
    d2 = np.array([0.0, 2.0, 1.0])
    # cell (i, j) has id 3*i + j and key d1[i] + d2[j]; by hand, sorted by (key, id):
    # id3 (1,0)=1 | id5 (1,2)=2, id6 (2,0)=2 | id0 (0,0)=3, id4 (1,1)=3, id8 (2,2)=3 | ...
    counts = np.array([1, 0, 2, 0, 3, 1, 1, 1, 1])
    cells, keys, total = O.traverse_full_sort(d1, d2, counts, 3)
    # counts along that order: 0, 1, 1, 1 -> prefix sums 0, 1, 2, 3: stop at id0
    assert cells.tolist() == [3, 5, 6, 0]
    assert keys.tolist() == [1.0, 2.0, 2.0, 3.0]
    assert total == 3
    cells, _, total = O.traverse_full_sort(d1, d2, counts, 4)
    assert cells.tolist() == [3, 5, 6, 0, 4] and total == 6


def test_visit_invariants():
    rng = np.random.default_rng(99)
    for _ in range(30):
        T = int(rng.integers(2, 30))
        d1, d2, counts = random_case(rng, T, ties=True)
        L = int(rng.integers(1, max(2, counts.sum() + 3)))
        cells, keys, total = O.traverse_multisequence(d1, d2, counts, L)
        ids = cells.tolist()
        # non-decreasing keys, ties broken by cell id
        assert all((keys[n], ids[n]) < (keys[n + 1], ids[n + 1]) for n in range(len(ids) - 1))
        # the candidate count and the shortest prefix
        assert total == int(counts[cells].sum())
        if counts.sum() >= L:
            assert total >= L and int(counts[cells[:-1]].sum()) < L
        else:
            assert len(ids) == T * T


def test_budget_must_be_positive():
    for walk in (O.traverse_full_sort, O.traverse_multisequence):
        with pytest.raises(ValueError):
            walk(np.zeros(2), np.zeros(2), np.ones(4, dtype=int), 0)


def test_single_coarse_codeword_is_one_list():
    """T = 1 reduces the multi-index to a single inverted list (IVF with one list)."""
    cells, keys, total = O.traverse_multisequence(np.array([4.0]), np.array([9.0]), np.array([7]), 3)
    assert cells.tolist() == [0] and total == 7 and keys.tolist() == [13.0]


def test_empty_cells_consume_order_but_not_budget():
    d1 = np.array([0.0, 10.0])
    d2 = np.array([0.0, 1.0])
    counts = np.array([0, 0, 5, 5])  # the two closest cells are empty
    cells, _, total = O.traverse_full_sort(d1, d2, counts, 1)
    assert cells.tolist() == [0, 1, 2] and total == 5
