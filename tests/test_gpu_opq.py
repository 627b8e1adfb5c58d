"""OPQ on the GPU (the optimized OMulti-D-OADC of §2.3) against the FP64 oracle.

Rotations make every vector real-valued, so the integer-grid exactness of the
plain path does not hold here; the readings checked instead:
* encoding: the GPU's cell and code of a point are the oracle's, except where the
  oracle's own distances tie within 1e-5 relative (FP32 rotation on the GPU);
* search on the same lists: distances within 1e-4 relative, ids equal except
  inside near-tie groups at the k-th rank (tests/parity.py);
* training: the GPU's learned rotations are orthogonal, diagonalize the learn
  set's covariance and deal balanced eigenvalue sums; given those rotations the
  oracle's training yields the GPU's codebooks bit for bit (integer grid after
  rounding).
"""
import numpy as np
import pytest

from oracle import bpq_oracle as O
from tests.parity import assert_topk_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def opq(tiny_oracle):
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    w = t["w"]
    cb = O.train_opq(t["learn"], w.T, w.M, 3)
    base = t["base"][:60_000]
    ix = bpq.Index.create(cb.C1, cb.C2, cb.R, rotations=(cb.rot0, cb.rot1, cb.rot2))
    ix.add(torch.as_tensor(base, dtype=torch.float32, device=DEV))
    ix.finalize()
    return dict(cb=cb, base=base, ix=ix)


def test_opq_encoding_matches_oracle_up_to_ties(opq):
    cb, base = opq["cb"], opq["base"][:20_000]
    x = torch.as_tensor(base, dtype=torch.float32, device=DEV)
    cells, codes = [t.cpu().numpy() for t in opq["ix"].encode(x)]
    o_cells, o_codes = O.encode_multi_d_adc(base, cb)
    same_cell = cells == o_cells
    assert same_cell.mean() > 0.999
    Xc = cb.coarse_space(base.astype(np.float64))
    h = cb.D // 2
    for n in np.nonzero(~same_cell)[0]:  # a different cell: a near-tie of the coarse distances
        for half, (C, a, b) in enumerate(((cb.C1, cells[n] // cb.T, o_cells[n] // cb.T),
                                          (cb.C2, cells[n] % cb.T, o_cells[n] % cb.T))):
            v = Xc[n, half * h:(half + 1) * h]
            da, db = ((v - C[a]) ** 2).sum(), ((v - C[b]) ** 2).sum()
            assert abs(da - db) <= 1e-5 * max(da, db, 1.0)
    ok = same_cell & (codes == o_codes).all(1)
    assert ok.mean() > 0.995


def test_opq_search_matches_oracle(opq, tiny_oracle):
    """The oracle searches the GPU's lists (checked above): FBPQ, the paper's tables and
    the reconstruction scorer agree with the oracle within tolerance."""
    cb = opq["cb"]
    a = opq["ix"].arrays()
    lists = O.Lists(T=cb.T, offsets=a["offsets"].cpu().numpy().astype(np.int64), codes=a["codes"].cpu().numpy(),
                    ids=a["ids"].cpu().numpy().astype(np.int64))
    oix = O.OracleIndex(cb=cb, lists=lists, variant="global", tables=O.fbpq_tables(cb))
    qn = tiny_oracle["queries"][:40]
    q = torch.as_tensor(qn, dtype=torch.float32, device=DEV)
    o_ids, o_d, _ = O.search(oix, qn, 5000, 50, "recon", traversal="full_sort")
    for scorer in ("fbpq", "fbpq_tables", "recon"):
        ids, d = opq["ix"].search(q, 5000, 50, scorer)
        assert_topk_match(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)


def test_opq_training_on_gpu(tiny_oracle):
    """GPU-learned rotations: orthogonal, diagonalizing, balanced; the oracle given
    them trains the same codebooks; the index searches like the oracle's."""
    import paper_1404_1831_gb300 as bpq
    t = tiny_oracle
    w = t["w"]
    learn = t["learn"]
    ix = bpq.Index.train(torch.as_tensor(learn, dtype=torch.float32, device=DEV), w.T, w.M, iters=3, opq=True)
    R0, R1, R2 = ix.rotations()
    for R in (R0, R1, R2):
        assert np.allclose(R @ R.T, np.eye(len(R)), atol=1e-9)
    X = learn.astype(np.float64)
    Xc = X - X.mean(0)
    C = R0 @ (Xc.T @ Xc / len(X)) @ R0.T
    assert np.abs(C - np.diag(np.diag(C))).max() < 1e-6 * np.abs(C).max()
    cb = O.train_opq(learn, w.T, w.M, 3, rotations=(R0, R1, R2))
    a = ix.arrays()
    for name in ("C1", "C2", "R"):
        assert np.array_equal(a[name].cpu().numpy(), getattr(cb, name).astype(np.float32)), name
    # OPQ lowers the learn set's encoding error against the plain codebooks
    plain = bpq.Index.train(torch.as_tensor(learn, dtype=torch.float32, device=DEV), w.T, w.M, iters=3)
    xl = torch.as_tensor(learn[:10_000], dtype=torch.float32, device=DEV)
    assert float(ix.encoding_error(xl).mean()) < float(plain.encoding_error(xl).mean())


def test_opq_save_load_and_shortlist(opq, tiny_oracle, tmp_path):
    import paper_1404_1831_gb300 as bpq
    path = tmp_path / "opq.bpq"
    opq["ix"].save(str(path))
    ix2 = bpq.Index.load(str(path))
    for A, B in zip(ix2.rotations(), opq["ix"].rotations()):
        assert np.array_equal(A, B)
    q = torch.as_tensor(tiny_oracle["queries"][:30], dtype=torch.float32, device=DEV)
    a = [x.cpu().numpy() for x in opq["ix"].search(q, 3000, 20, "fbpq")]
    b = [x.cpu().numpy() for x in ix2.search(q, 3000, 20, "fbpq")]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = [x.cpu().numpy() for x in opq["ix"].search_shortlist(q, 3000, 20, shortlist=200, precision="fp16")]
    assert np.array_equal(a[0], c[0])
