"""Host side of the serving loop: the seeded Poisson arrival process."""
import numpy as np

from paper_1404_1831_gb300 import serving


def test_poisson_arrivals_rate_and_order():
    a = serving.poisson_arrivals(200_000, 50_000.0, 3)
    assert np.all(np.diff(a) > 0)
    gaps = np.diff(np.concatenate([[0.0], a]))
    # exponential gaps: mean 1/rate, standard deviation 1/rate (relative error of the mean ~ 1/sqrt(n))
    assert abs(gaps.mean() * 50_000.0 - 1.0) < 0.01
    assert abs(gaps.std() * 50_000.0 - 1.0) < 0.02
    # counts in unit windows are Poisson: variance equals mean
    counts = np.bincount((a * 1000).astype(np.int64))[:-1]
    assert abs(counts.var() / counts.mean() - 1.0) < 0.1


def test_poisson_arrivals_seeded():
    assert np.array_equal(serving.poisson_arrivals(100, 10.0, 7), serving.poisson_arrivals(100, 10.0, 7))
    assert not np.array_equal(serving.poisson_arrivals(100, 10.0, 7), serving.poisson_arrivals(100, 10.0, 8))
