"""Host logic of bench.py: the digest that keys recorded DRAM counters to kernel code."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_source_digest_ignores_comments_but_not_code(tmp_path):
    b = _bench()
    base = "// header\n__global__ void k(int* p) {\n  p[0] = 1;  // store\n}\n"
    f = tmp_path / "k.cu"
    f.write_text(base)
    d0 = b.source_digest(str(f))
    f.write_text("/* a new\n   block comment */\n" + base.replace("// store", "// the store") + "\n\n")
    assert b.source_digest(str(f)) == d0
    f.write_text(base.replace("p[0] = 1;", "p[0] = 2;"))
    assert b.source_digest(str(f)) != d0


def test_recorded_counters_match_the_current_kernels():
    """profiles/traffic.json carries the digest of the code its counters were taken on;
    the bench reports them only while that digest still matches."""
    b = _bench()
    for f in ("bpq_scan.cu", "bpq_traverse.cu"):
        rec = b.recorded_traffic(f)
        assert rec is None or rec["source_sha256_16"] == b.source_digest(
            os.path.join(ROOT, "paper_1404_1831_gb300", "csrc", f))


def test_launch_claim_counts_every_kernel_of_a_search():
    """The bench's gpu_launches claim: two table kernels (coarse and PQ) for the FBPQ scorers, the
    traversal's two passes at T <= 1024, and two scan launches for the FBPQ per-point scorer with
    k <= 128 (the finished queries, and on the second stream the handed-over ones)."""
    import dataclasses

    import synthdata as sd
    b = _bench()
    w = sd.SIFT10M
    assert b.launches_per_step(w, "fbpq", 100) == 6
    assert b.launches_per_step(w, "fbpq", 1000) == 5
    assert b.launches_per_step(w, "fbpq_tables", 100) == 5
    assert b.launches_per_step(w, "recon", 100) == 4
    big_T = dataclasses.replace(w, T=2048)
    assert b.launches_per_step(big_T, "fbpq", 100) == 4
