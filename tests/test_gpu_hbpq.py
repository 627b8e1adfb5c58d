"""GPU parity for HBPQ (§3.2): local codebook training, local encoding and the
HBPQ scorer against the FP64 oracle, on a reduced tiny workload."""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hbpq(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    w = t["w"]
    iters = 4
    cb = O.train_multi_d_adc(t["learn"], w.T, w.M, iters)
    cbl = O.train_hbpq_local(t["learn"], cb, iters)
    base = t["base"][:40_000]
    oix = O.build_index(cbl, base, variant="local")
    learn = torch.as_tensor(t["learn"], dtype=torch.float32, device=DEV)
    ix = bpq.Index.train(learn, w.T, w.M, variant="local", iters=iters)
    ix.add(torch.as_tensor(base, dtype=torch.float32, device=DEV))
    ix.finalize()
    return dict(ix=ix, oix=oix, cbl=cbl, base=base)


def test_local_training_bit_exact(hbpq):
    a = hbpq["ix"].arrays()
    assert np.array_equal(a["Q"].cpu().numpy(), hbpq["cbl"].Q.astype(np.float32))
    assert np.array_equal(a["S"].cpu().numpy(), hbpq["cbl"].S.astype(np.float32))


def test_local_encoding_bit_exact(hbpq):
    a = hbpq["ix"].arrays()
    assert np.array_equal(a["codes"].cpu().numpy(), hbpq["oix"].lists.codes)
    assert np.array_equal(a["offsets"].cpu().numpy().astype(np.int64), hbpq["oix"].lists.offsets)


def test_hbpq_search_matches_oracle(hbpq, tiny_oracle):
    qn = tiny_oracle["queries"][:40]
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    ids, d = hbpq["ix"].search(q, 4000, 50, "hbpq")
    o_ids, o_d, _ = O.search(hbpq["oix"], qn, 4000, 50, "hbpq")
    assert assert_topk_match(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d) == len(qn)
