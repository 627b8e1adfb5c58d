"""Points added twice under the same id (bpq_add accepts any ids >= 0).

Both copies land in the same cell with the same code, so they get the same
distance and the same id: equal (distance, id) composites.  Every scorer must
return both copies, in consecutive ranks, exactly as the oracle's stable ranking
does, and never leave a result slot unwritten."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def dup(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    cb = tiny_oracle["cb"]
    base = tiny_oracle["base"][:6000]
    X = np.concatenate([base, base[:3000]])
    ids = np.concatenate([np.arange(6000), np.arange(3000)]).astype(np.int32)
    oix = O.build_index(cb, X, ids=ids)
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R)
    ix.add(torch.as_tensor(X, dtype=torch.float32, device=DEV), ids=torch.as_tensor(ids, device=DEV))
    ix.finalize()
    return ix, oix


@pytest.mark.parametrize("scorer", ["fbpq", "fbpq_tables", "recon"])
@pytest.mark.parametrize("k", [10, 100, 300])
def test_duplicated_ids_are_both_returned(dup, tiny_oracle, scorer, k):
    ix, oix = dup
    qn = tiny_oracle["queries"][:16]
    # poison the output buffers: a slot the kernel does not write keeps the marker
    ids = torch.full((len(qn), k), -7, dtype=torch.int32, device=DEV)
    dists = torch.full((len(qn), k), -7.0, dtype=torch.float32, device=DEV)
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    ix.search(q, 2000, k, scorer, out=(ids, dists))
    g_ids, g_d = ids.cpu().numpy(), dists.cpu().numpy()
    assert not (g_ids == -7).any()
    o_ids, o_d, _ = O.search(oix, qn, 2000, k, "fbpq")
    assert assert_topk_match(g_ids, g_d, o_ids, o_d) == len(qn)
    # the duplicates really occur in the answers
    assert any(len(set(r.tolist())) < len(r) for r in g_ids)
