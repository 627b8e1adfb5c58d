"""bpq_search_noalloc: the search for callers that must not allocate device memory.

Programs that hand all GPU memory to their own pool, or serving loops where a
cudaMalloc / cudaFree (which can stall the whole device) is not allowed, cannot
give bpq_search a workspace.  bpq_search_noalloc runs the same kernels with the
library's built-in scratch array instead.  These tests call it through the C ABI
twice in a row and check each result against bpq_search, within the tolerance
used by the other parity tests.  The file is named so that pytest collects it
last; it builds its own small index, so it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def small_index():
    import paper_1404_1831_gb300 as bpq
    import synthdata as sd
    mix = sd.make_mixture(2024, 32)
    learn = torch.as_tensor(sd.points(mix, sd.STREAM_LEARN, 0, 8000), dtype=torch.float32, device=DEV)
    ix = bpq.Index.train(learn, 64, 8, iters=5)
    ix.add(torch.as_tensor(sd.points(mix, sd.STREAM_BASE, 0, 60_000), dtype=torch.float32, device=DEV))
    ix.finalize()
    q = torch.as_tensor(sd.points(mix, sd.STREAM_QUERY, 0, 64), dtype=torch.float32, device=DEV)
    return ix, q


def test_two_noalloc_calls_match_bpq_search(small_index):
    ix, q = small_index
    status = torch.full((1,), 7, dtype=torch.int32, device=DEV)
    # first call: one budget for every query, FBPQ scoring
    a_ids, a_d = ix.search_noalloc(q, 6000, 100, "fbpq", status=status)
    r_ids, r_d = ix.search(q, 6000, 100, "fbpq")
    assert_topk_match(a_ids.cpu().numpy(), a_d.cpu().numpy(), r_ids.cpu().numpy(), r_d.cpu().numpy())
    assert int(status.item()) == 0
    # second call right after it, reusing the same built-in scratch: a budget per
    # query and the reconstruction scorer
    Ls = np.random.default_rng(3).integers(50, 20_000, size=q.shape[0])
    b_ids, b_d = ix.search_noalloc(q, Ls, 37, "recon", status=status)
    s_ids, s_d = ix.search(q, Ls, 37, "recon")
    assert_topk_match(b_ids.cpu().numpy(), b_d.cpu().numpy(), s_ids.cpu().numpy(), s_d.cpu().numpy())
    assert int(status.item()) == 0


def test_batch_larger_than_the_scratch_is_rejected(small_index):
    import paper_1404_1831_gb300 as bpq
    ix, q = small_index
    big = q.repeat(200, 1)  # 12,800 queries at L = 50,000: far beyond the built-in scratch
    need = bpq.lib().bpq_search_workspace_size(ix._h, big.shape[0], 50_000, 10, 0)
    assert need > bpq.lib().bpq_search_workspace_size(ix._h, 1, 50_000, 10, 0)
    with pytest.raises(bpq.BpqError) as e:
        ix.search_noalloc(big, 50_000, 10)
    assert e.value.code == -7
