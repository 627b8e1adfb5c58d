import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload, minutes of host time")


@pytest.fixture(scope="session")
def tiny_oracle():
    """Tiny workload (100k points, T=64, M=8) built once by the oracle."""
    import synthdata as sd
    from oracle import bpq_oracle as O
    w = sd.TINY
    mix = sd.make_mixture(w.seed, w.n_comp, w.dim)
    learn = sd.points(mix, sd.STREAM_LEARN, 0, w.n_learn)
    base = sd.points(mix, sd.STREAM_BASE, 0, w.n_base)
    queries = sd.points(mix, sd.STREAM_QUERY, 0, w.n_query)
    cb = O.train_multi_d_adc(learn, w.T, w.M, w.kmeans_iters)
    index = O.build_index(cb, base)
    return dict(w=w, mix=mix, learn=learn, base=base, queries=queries, cb=cb, index=index)
