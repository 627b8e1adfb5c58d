#!/usr/bin/env python
"""Throughput benchmark of the bilayer product-quantization search path on GB300.

Workload (synthetic, SIFT-shaped, generated on the device from synthdata):
10,000,000 points of dimension 128 (integer coordinates in [0, 255]), an inverted
multi-index with T = 1024 coarse codewords per half (1,048,576 cells), M = 8
residual PQ codes of 256 codewords, codebooks trained on the GPU with 10 Lloyd
iterations on 1,024,000 learn points; 10,000 queries per step at candidate
budget L = 10,000, top-100 returned, FBPQ scoring.

One step = bpq_search over the 10,000 queries (query tables, traversal, scan,
top-k) with queries, index and workspace resident in HBM.  L2 (129 MB) is flushed
between steps by writing a 512 MB buffer outside the timed events.

  python bench.py [--gpus N --steps K --warmup W]      our CUDA path (torchrun for N > 1)
  python bench.py --impl reference ...                 the FP64 CPU oracle on the host cores

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s at fixed L & Recall@10, FBPQ vs reconstruct-ADC; p50/p99 serve latency"
UNIT = "queries/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--L", type=int, default=10_000)
    ap.add_argument("--k", type=int, default=100)
    ap.add_argument("--scorer", default="fbpq")
    ap.add_argument("--n-base", type=int, default=None, help="override the point count (testing only)")
    ap.add_argument("--n-query", type=int, default=None, help="override the queries per step (profiling only)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the L / scorer sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the Poisson serving measurement")
    ap.add_argument("--no-configs", action="store_true", help="skip the 100M / 1B configuration blocks")
    ap.add_argument("--workload", choices=("sift10m", "c3", "c4", "c5", "gist", "opq"), default="sift10m",
                    help="c3: 100M, M=16, int8 shortlist; c4: 100M, local codebooks, uneven L; "
                         "c5: 1B points, serving (each prints its own JSON line)")
    ap.add_argument("--serve-seconds", type=float, default=0.25, help="arrival window per offered load")
    ap.add_argument("--oracle-seconds", type=float, default=12.0)
    return ap.parse_args()


def workload(args):
    import dataclasses

    import synthdata as sd
    w = sd.SIFT10M
    if args.n_base:
        w = dataclasses.replace(w, n_base=args.n_base)
    if args.n_query:
        w = dataclasses.replace(w, n_query=args.n_query)
    return w


# ---------------------------------------------------------------------------
# Oracle (CPU) side: runs in spawned processes only.
# ---------------------------------------------------------------------------
ORACLE_LEARN = 100_000
ORACLE_ITERS = 4


def _oracle_encode_chunk(task):
    import synthdata as sd
    from oracle import bpq_oracle as O
    seed, n_comp, start, count, cb = task
    mix = sd.make_mixture(seed, n_comp)
    x = sd.points(mix, sd.STREAM_BASE, start, count)
    return O.encode_multi_d_adc(x, cb)


_ORACLE_INDEX = None  # the timing processes' index (inherited by fork from the oracle worker)


def _oracle_time_slice(task):
    """Times the oracle's search of queries [a, b) (one process, one core)."""
    import synthdata as sd
    from oracle import bpq_oracle as O
    w, L, k, a, b, seconds = task
    mix = sd.make_mixture(w.seed, w.n_comp)
    queries = sd.points(mix, sd.STREAM_QUERY, a, b - a)
    O.search_one(_ORACLE_INDEX, queries[0], L, k, "fbpq")  # warm caches
    times, t1 = [], time.time()
    for n in range(b - a):
        if time.time() - t1 >= seconds:
            break
        s0 = time.time()
        O.search_one(_ORACLE_INDEX, queries[n], L, k, "fbpq")
        times.append(time.time() - s0)
    return times


def _oracle_worker(w, L, k, seconds, nq_max, out_q, procs, cb_arrays):
    """Builds the oracle's index of the workload (with the given codebooks, else its own
    training), then times its search on one core and on `procs` cores at once.  Runs in a
    spawned process that never touches the GPU, so it may fork its timing processes."""
    global _ORACLE_INDEX
    import numpy as np

    import synthdata as sd
    from oracle import bpq_oracle as O
    t0 = time.time()
    mix = sd.make_mixture(w.seed, w.n_comp)
    if cb_arrays is not None:
        cb = O.Codebooks(D=w.dim, T=w.T, M=w.M, **{n: np.asarray(v, dtype=np.int64) for n, v in cb_arrays.items()})
    else:
        learn = sd.points(mix, sd.STREAM_LEARN, 0, min(ORACLE_LEARN, w.n_learn))
        cb = O.train_multi_d_adc(learn, w.T, w.M, ORACLE_ITERS)
    step = 250_000
    tasks = [(w.seed, w.n_comp, s, min(step, w.n_base - s), cb) for s in range(0, w.n_base, step)]
    with mp.get_context("fork").Pool(procs) as pool:
        parts = pool.map(_oracle_encode_chunk, tasks)
    cells = np.concatenate([p[0] for p in parts])
    codes = np.concatenate([p[1] for p in parts])
    _ORACLE_INDEX = O.OracleIndex(cb=cb, lists=O.build_lists(cells, codes, np.arange(w.n_base), w.T),
                                  variant="global", tables=O.fbpq_tables(cb))
    build_s = time.time() - t0
    one = _oracle_time_slice((w, L, k, 0, nq_max, seconds))
    res = dict(n=len(one), seconds=sum(one), times=one, build_s=build_s)
    if procs > 1:  # P processes over disjoint query slices, all at once: aggregate queries/s
        per = 100
        slices = [(w, L, k, nq_max + i * per, nq_max + (i + 1) * per, seconds) for i in range(procs)]
        t1 = time.time()
        with mp.get_context("fork").Pool(procs) as pool:
            parts = pool.map(_oracle_time_slice, slices)
        wall = time.time() - t1
        res["multi"] = dict(procs=procs, queries=sum(len(p) for p in parts), wall_s=wall)
    out_q.put(res)


def run_oracle(w, L, k, seconds, nq_max=200, cb_arrays=None, multi=True):
    """Oracle search timing in a spawned process with single-threaded BLAS."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    saved = {v: os.environ.get(v) for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in saved:
        os.environ[v] = "1"
    procs = max(1, min(16, os.cpu_count() or 1))
    try:
        p = ctx.Process(target=_oracle_worker,
                        args=(w, L, k, seconds, nq_max, q, procs if multi else 1, cb_arrays))
        p.start()
        res = q.get()
        p.join()
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    return res


def oracle_sample_text(w, L, n, own=True):
    cbs = (f"the oracle's own codebooks ({ORACLE_ITERS} Lloyd iterations on {ORACLE_LEARN} learn points)" if own
           else "the GPU arm's codebooks (the same index)")
    return (f"{n} queries of the {w.name} workload (N={w.n_base}, T={w.T}, M={w.M}) at L={L}, k=100, FBPQ "
            f"scoring, one at a time on one core, on the oracle's lists built with {cbs}")


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------
def launches_per_step(w, scorer, k=100):
    """Kernels one search launches: the query tables (one more for the LUT of the
    table-based scorers), the traversal (its common path and the fallback pass
    when T <= 1024) and the scan (twice for the FBPQ per-point scorer with k <= 128
    and T <= 1024: the queries the common traversal path finished, and on the
    second stream the ones it handed over)."""
    tables = 2 if scorer in ("fbpq", "fbpq_tables") else 1
    traverse = 2 if w.T <= 1024 else 1
    scans = 2 if (scorer == "fbpq" and k <= 128 and w.T <= 1024) else 1
    return tables + traverse + scans


class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        self.marks = {}

    def mark(self, name):
        self.marks[name] = time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.tmp.flush()
        rows = []
        for line in open(self.tmp.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append(dict(ts=ts, sm=float(parts[2]), smax=float(parts[3]), power=parts[4],
                                 hw=parts[6], hwt=parts[7], swt=parts[8], swp=parts[9]))
            except ValueError:
                continue
        os.unlink(self.tmp.name)
        t0, t1 = self.marks.get("start", 0), self.marks.get("end", 1e18)
        inside = [r for r in rows if t0 - 0.15 <= r["ts"] <= t1 + 0.15]
        window = "timed region"
        if not inside:
            inside, window = rows, "warm-up and timed region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = set()
        for r in inside:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in inside), "sm_max_mhz": max(r["smax"] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


def source_digest(path):
    """Digest of a source file's code: comments, blank lines and trailing blanks are left out, so a
    comment edit keeps the recorded counters of an unchanged kernel."""
    import re
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()[:16]


def recorded_traffic(kernel_file):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    src = os.path.join(ROOT, "paper_1404_1831_gb300", "csrc", kernel_file)
    ent = rec.get(kernel_file)
    if ent and ent.get("source_sha256_16") == source_digest(src):
        return ent
    return None


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.backends.cuda.matmul.allow_tf32 = False

    import paper_1404_1831_gb300 as bpq
    from paper_1404_1831_gb300 import multi
    import synthdata as sd
    from synthdata import device as sdev

    w = workload(args)
    want_cpu = (rank == 0 and world == 1 and not args.no_cpu_baseline)
    t_setup = time.time()
    mix = sd.make_mixture(w.seed, w.n_comp)
    learn = sdev.points_cuda(mix, sd.STREAM_LEARN, 0, w.n_learn, device=dev)
    ix = bpq.Index.train(learn, w.T, w.M, iters=w.kmeans_iters)
    del learn
    chunk = 2_000_000
    for s in range(0, w.n_base, chunk):
        x = sdev.points_cuda(mix, sd.STREAM_BASE, s, min(chunk, w.n_base - s), device=dev)
        ix.add(x)
        del x
    ix.finalize()
    info = ix.info()
    nq = w.n_query
    q0, _ = multi.replica_queries(rank, nq)  # replicas: every rank answers its own batch
    queries = sdev.points_cuda(mix, sd.STREAM_QUERY, q0, nq, device=dev)
    torch.cuda.synchronize()
    setup_s = time.time() - t_setup

    L, k, scorer = args.L, args.k, args.scorer
    ws = ix.workspace(nq, L, k, scorer)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return ix.search(queries, L, k, scorer, workspace=ws)

    # per-phase kernel times (the same kernels bpq_search launches), CUDA events on this stream
    cap = int(min(L, max(1, info.n_nonempty)))
    cells = torch.empty((nq, cap, 4), dtype=torch.int32, device=dev)
    ncells = torch.empty(nq, dtype=torch.int32, device=dev)
    npts = torch.empty(nq, dtype=torch.int64, device=dev)
    tws = ix.workspace(nq, L, k, scorer)

    def phases(reps=3):
        res = {"tables": [], "traverse": [], "scan": []}
        for _ in range(reps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            d1, d2, lut = ix.query_tables(queries, lut=scorer.startswith("fbpq"))
            ev[1].record(stream)
            Ls, stride = bpq._L_array(L, nq)
            bpq._check(bpq.lib().bpq_traverse(ix._h, bpq._ptr(queries), nq, Ls.ctypes.data, stride, cap,
                                              bpq._ptr(cells), bpq._ptr(ncells), bpq._ptr(npts), bpq._ptr(tws),
                                              tws.numel(), bpq._stream()))
            ev[2].record(stream)
            ix.scan(queries, lut, cells, ncells, k, scorer)
            ev[3].record(stream)
            torch.cuda.synchronize()
            res["tables"].append(ev[0].elapsed_time(ev[1]))
            res["traverse"].append(ev[1].elapsed_time(ev[2]))
            res["scan"].append(ev[2].elapsed_time(ev[3]))
        return {kk: statistics.median(v) for kk, v in res.items()}

    for _ in range(max(1, args.warmup)):
        step()
    ph = phases()
    cand = int(npts.sum().item())
    ncell_total = int(ncells.clamp(min=0).sum().item())

    # main timed region
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark("start")
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler.mark("end")
    clocks = sampler.stop()
    ix.search_status(ws)
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = multi.max_over_ranks(total_ms, device=dev)
    value = nq * world * args.steps / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    qh = torch.empty((nq, w.dim), dtype=torch.float32).pin_memory()
    qh.copy_(queries.cpu())
    idsh = torch.empty((nq, k), dtype=torch.int32).pin_memory()
    dh = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    Ls, stride = bpq._L_array(L, nq)

    def e2e_step():
        bpq._check(bpq.lib().bpq_search_host(ix._h, qh.data_ptr(), nq, Ls.ctypes.data, stride, k,
                                             bpq.SCORERS[scorer], idsh.data_ptr(), dh.data_ptr(), bpq._stream()))

    for _ in range(max(1, args.warmup)):
        e2e_step()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = sum(e2e_ms)
    if world > 1:
        e2e_total = multi.max_over_ranks(e2e_total, device=dev)
    e2e = {"value": nq * world * args.steps / (e2e_total / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": nq * w.dim * 4, "d2h_bytes_per_step": nq * k * 8,
           "ms_per_step": e2e_total / args.steps}

    # roofline of the dominant kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # The dominant kernel: the scan is one launch; the traversal phase is two kernels (the warp
    # pass and the CTA pass over the queries it hands over), each shorter than the phase.  The
    # scan is therefore reported whenever its phase is at least half the traversal phase (the
    # launch list under profiles/ gives the per-kernel shares); the traversal phase is reported
    # beside it.
    scan_bytes = cand * (w.M + 4)
    trav_bytes = ncell_total * 16 + nq * 2 * w.T * 4
    tr_s, tr_t = recorded_traffic("bpq_scan.cu"), recorded_traffic("bpq_traverse.cu")
    kname = "fbpq_scan_seg_kernel" if scorer == "fbpq" and k <= 128 else f"{scorer}_scan_kernel"
    roof_scan = {"kernel": kname, "bound": "hbm", "achieved": scan_bytes / (ph["scan"] / 1e3) / 1e9,
                 "peak": hbm_peak, "unit": "GB/s", "peak_source": peak_src,
                 "algorithmic_bytes_per_launch": scan_bytes, "bytes_per_candidate": w.M + 4,
                 # DRAM bytes of a smaller captured launch, scaled by the units this launch processes
                 "traffic": tr_s["bytes_per_candidate"] * cand if tr_s else None,
                 "traffic_source": tr_s["source"] if tr_s else None}
    roof_trav = {"kernel": "traverse_warp_kernel + traverse_kernel", "bound": "hbm",
                 "achieved": trav_bytes / (ph["traverse"] / 1e3) / 1e9,
                 "peak": hbm_peak, "unit": "GB/s", "peak_source": peak_src,
                 "algorithmic_bytes_per_launch": trav_bytes,
                 "traffic": tr_t["bytes_per_query"] * nq if tr_t else None,
                 "traffic_source": tr_t["source"] if tr_t else None,
                 "note": "latency-bound (per-query sorts and band searches); bytes = cell records written + coarse tables read"}
    for r in (roof_scan, roof_trav):
        r["frac"] = r["achieved"] / r["peak"]
    scan_dominant = ph["scan"] >= 0.5 * ph["traverse"]
    roof = roof_scan if scan_dominant else roof_trav

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "n_base": w.n_base, "dim": w.dim, "T": w.T, "M": w.M, "n_query": nq,
                      "L": L, "k": k, "scorer": scorer, "codebooks": f"GPU k-means, {w.kmeans_iters} Lloyd "
                      f"iterations on {w.n_learn} learn points", "l2": "flushed between steps (512 MB write)",
                      "parallelism": f"replicas x{world} (independent query batches)"},
           "roofline": roof, "roofline_other": roof_trav if scan_dominant else roof_scan,
           "gpu_launches": launches_per_step(w, scorer, k) * args.steps, "clocks": clocks,
           "phases_ms": ph, "candidates_per_step": cand, "visited_cells_per_step": ncell_total,
           "index": {"n_points": info.n_points, "n_nonempty_cells": info.n_nonempty, "max_cell": info.max_cell},
           "e2e": e2e, "setup_s": round(setup_s, 1)}

    if rank == 0 and world == 1 and not args.no_sweep:
        out["sweep"] = sweep(ix, queries, w, k, flush, stream)
        out["recall"] = recall(ix, queries, w, mix, L, k, dev)
        out["batching"] = {"timing": "host wall time per batch over 50 back-to-back launches",
                           "shapes": [batching_block(ix, queries[:nb].clone(), Lb, k, scorer)
                                      for nb, Lb in ((16, 1_000), (64, 10_000), (64, 100_000), (512, 100_000))]}
    if rank == 0 and world == 1 and not args.no_serve:
        out["serve"] = serve_block(ix, w, mix, k, args.serve_seconds)

    cb_arrays = None
    if want_cpu:  # the CPU baseline searches the same index: the GPU arm's codebooks
        a = ix.arrays()
        cb_arrays = {n: a[n].cpu().numpy() for n in ("C1", "C2", "R")}
        del a
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    del ix, ws, tws, cells, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_configs:
        # the 100M and 1B configurations, each on a fresh index (outside the timed region)
        out["configs"] = {}
        for name in ("c3", "c4", "c5", "gist", "opq"):
            t0 = time.time()
            out["configs"][name] = config_block(name, args.serve_seconds)
            out["configs"][name]["wall_s"] = round(time.time() - t0, 1)
            torch.cuda.empty_cache()
    if want_cpu:
        res = run_oracle(w, L, k, args.oracle_seconds, cb_arrays=cb_arrays)
        out["cpu_baseline"] = {"value": res["n"] / res["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": oracle_sample_text(w, L, res["n"], own=False),
                               "same_codebooks_as_gpu": True,
                               "ms_per_query_median": 1e3 * statistics.median(res["times"]),
                               "oracle_index_build_s": round(res["build_s"], 1)}
        if "multi" in res:
            m = res["multi"]
            out["cpu_baseline"]["all_cores"] = {
                "value": m["queries"] / m["wall_s"], "unit": UNIT, "cores": m["procs"],
                "sample": f"{m['procs']} processes at once, each timing its own slice of the query stream "
                          f"(disjoint queries), for about {args.oracle_seconds:.0f} s; aggregate queries/s"}
    if rank == 0:
        print(json.dumps(out), flush=True)


def serve_block(ix, w, mix, k, seconds, seed=11, n_max=300_000, max_batch=4096, slots=3, device_bytes=12 << 30):
    """Poisson stream with per-query L uniform over {1k, 10k, 100k}, latency from arrival to results in host
    memory.  Continuous batching (bpq_server: `slots` batches in flight on their own streams, admission by
    device memory, one budget class per batch) at 50 % and 80 % of its saturated throughput (every query
    queued at time zero), next to the blocking queue (one bpq_search_host call at a time) at the same
    offered rates."""
    import numpy as np
    import torch

    import synthdata as sd
    from paper_1404_1831_gb300 import serving
    from synthdata import device as sdev
    qh = sdev.points_cuda(mix, sd.STREAM_QUERY, w.n_query, n_max).cpu().numpy()  # after the timed batch
    mix_L = np.array([1_000, 10_000, 100_000], dtype=np.int64)
    Ls = mix_L[np.random.default_rng(seed).integers(0, len(mix_L), n_max)]
    n_sat = min(n_max, 120_000)
    # scan schedule per batch class the server will form (budget class x batch size), by measurement
    qd = torch.as_tensor(qh[:max_batch], device="cuda")
    tuned = {f"L{int(Lc)}_n{nb}": ix.autotune(qd[:nb], int(Lc), k)
             for Lc in mix_L for nb in (32, 128, 512, 2048)}
    cfg = dict(k=k, slots=slots, max_batch=max_batch, L_max=int(mix_L.max()), device_bytes=device_bytes)
    serving.serve_continuous(ix, qh[:4096], Ls[:4096], np.zeros(4096), **cfg)  # warm-up
    # saturated rate: every query queued at time zero; the better of two passes (a pass lasts tens of
    # milliseconds, so one host-side hiccup would otherwise set the offered loads below)
    sat = min((serving.serve_continuous(ix, qh[:n_sat], Ls[:n_sat], np.zeros(n_sat), **cfg) for _ in range(2)),
              key=lambda r: r.wall_s)
    sat_qps = n_sat / sat.wall_s
    sat_queue = serving.saturated_qps(ix, qh, Ls, k, batch=max_batch)
    out = {"L_mix": mix_L.tolist(), "k": k, "latency": "arrival to results in host memory (copies included)",
           "continuous": {"slots": slots, "max_batch": max_batch, "device_bytes": device_bytes,
                          "admission": "bpq_search_workspace_size of the batch at its largest L <= device_bytes / slots",
                          "batching": "one budget class (floor(log2 L)) per batch, oldest class first",
                          "autotuned_work_items": tuned,
                          "saturated_qps": sat_qps, "saturated_stats": sat.stats, "loads": {}},
           "queue": {"max_batch": max_batch, "saturated_qps": sat_queue, "loads": {}}}
    for load in (0.5, 0.8):
        rate = load * sat_qps
        n = int(min(n_max, max(1000, rate * seconds)))
        arr = serving.poisson_arrivals(n, rate, seed + int(10 * load))
        res = serving.serve_continuous(ix, qh[:n], Ls[:n], arr, **cfg)
        out["continuous"]["loads"][f"{load:.1f}"] = {"offered_qps": rate, **res.summary(),
                                                     "max_in_flight": res.stats["max_in_flight"]}
        res = serving.serve(ix, qh[:n], Ls[:n], arr, k, max_batch=max_batch)
        out["queue"]["loads"][f"{load:.1f}"] = {"offered_qps": rate, **res.summary()}
    return out


def sweep(ix, queries, w, k, flush, stream, steps=3):
    """Queries/s of FBPQ and reconstruction-ADC at each budget of the workload."""
    import torch
    res = {}
    nq = queries.shape[0]
    for L in w.L:
        for scorer in ("fbpq", "fbpq_tables", "recon"):
            ws = ix.workspace(nq, L, k, scorer)
            ix.search(queries, L, k, scorer, workspace=ws)
            ms = []
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ix.search(queries, L, k, scorer, workspace=ws)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            res[f"{scorer}_L{L}"] = {"qps": nq / (statistics.median(ms) / 1e3), "ms": statistics.median(ms)}
        res[f"speedup_L{L}"] = res[f"fbpq_L{L}"]["qps"] / res[f"recon_L{L}"]["qps"]
        res[f"speedup_tables_L{L}"] = res[f"fbpq_tables_L{L}"]["qps"] / res[f"recon_L{L}"]["qps"]
    return res


def batching_block(ix, q, L, k, scorer, reps=50):
    """One batch shape three ways, host wall time per batch (launches included): bpq_search; the same
    search as one CUDA-graph launch; the graph of the autotuned scan schedule (bpq_autotune)."""
    import torch
    nq = q.shape[0]
    Ls = L if hasattr(L, "__len__") else int(L)
    ws = ix.workspace(nq, int(max(L) if hasattr(L, "__len__") else L), k, scorer)

    def wall(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    t_search = wall(lambda: ix.search(q, Ls, k, scorer, workspace=ws))
    g = ix.graph(q, Ls, k, scorer)
    t_graph = wall(g.launch)
    g.close()
    W = ix.autotune(q, Ls, k, scorer)
    g = ix.graph(q, Ls, k, scorer)
    t_tuned = wall(g.launch)
    g.close()
    return {"nq": nq, "search_ms": t_search, "graph_ms": t_graph, "autotuned_work_item": W,
            "autotuned_graph_ms": t_tuned}


def exact_nn_gpu(q, w, mix, dev, chunk=2_000_000):
    """Exact nearest neighbour of each query over the base points, by brute force with TF32 off: the inner
    products are taken over blocks of at most 128 dimensions in FP32 (integer data in [0, 255]: every
    partial sum is an integer below 2^24, so exact) and added in FP64."""
    import torch

    import synthdata as sd
    from synthdata import device as sdev
    n = q.shape[0]
    D = q.shape[1]
    wide = D > 128
    chunk = chunk // 4 if wide else chunk
    ft = torch.float64 if wide else torch.float32
    qn = (q.to(ft) * q.to(ft)).sum(1, keepdim=True)
    best = torch.full((n,), float("inf"), dtype=ft, device=dev)
    arg = torch.zeros(n, dtype=torch.int64, device=dev)
    for s in range(0, w.n_base, chunk):
        x = sdev.points_cuda(mix, sd.STREAM_BASE, s, min(chunk, w.n_base - s), device=dev)
        dot = sum((q[:, b:b + 128] @ x[:, b:b + 128].T).to(ft) for b in range(0, D, 128))
        d = qn - 2.0 * dot + (x.to(ft) * x.to(ft)).sum(1)[None, :]
        m, a = d.min(1)
        upd = m < best
        best = torch.where(upd, m, best)
        arg = torch.where(upd, a + s, arg)
    return arg


def recall_of(ids, nn):
    hit = (ids.long() == nn[:, None])
    return {f"R@{R}": float(hit[:, :R].any(1).float().mean()) for R in (1, 10, 100)}


def config_block(name, serve_seconds=0.25):
    """One of the larger configurations, measured on the GPU (returns a dict):
      c3  100M points, M = 16, L = 30k: FP32 FBPQ vs the int8 and FP16 table shortlists (1000) with exact
          re-scoring; identical-list fraction, recall;
      c4  100M points, L = round(10^U(3, 5)) per query: HBPQ (tables on the tensor cores, and the O(D)
          reconstruction) vs the global codebooks' FBPQ and reconstruction; recall;
      c5  1B points: FBPQ batch queries/s at L = 1k / 10k / 100k, resident bytes of both FBPQ forms, and
          continuous-batching serving latency.
    Recall is against exact nearest neighbours by GPU brute force (1,000 queries).  Oracle parity at these
    sizes is checked by the slow GPU tests, not here."""
    import numpy as np
    import torch

    import paper_1404_1831_gb300 as bpq
    import synthdata as sd
    from synthdata import device as sdev
    dev = torch.device("cuda", 0)
    torch.backends.cuda.matmul.allow_tf32 = False
    w = {"c3": sd.SIFT100M_M16, "c4": sd.SIFT100M, "c5": sd.SIFT1B, "gist": sd.GIST50M, "opq": sd.SIFT10M}[name]
    mix = sd.make_mixture(w.seed, w.n_comp, w.dim)
    learn = sdev.points_cuda(mix, sd.STREAM_LEARN, 0, w.n_learn, device=dev)

    def build(variant, opq=False):
        t0 = time.time()
        ix = bpq.Index.train(learn, w.T, w.M, variant=variant, iters=w.kmeans_iters, opq=opq)
        for s in range(0, w.n_base, 4_000_000):
            ix.add(sdev.points_cuda(mix, sd.STREAM_BASE, s, min(4_000_000, w.n_base - s), device=dev))
        ix.finalize()
        torch.cuda.synchronize()
        return ix, time.time() - t0

    q = sdev.points_cuda(mix, sd.STREAM_QUERY, 0, w.n_query, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=5, warm=3):
        ts = []
        for r in range(warm + reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= warm:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def enc_error(ix, n=10_000_000):
        """Mean squared encoding error ||x - xhat||^2 over the first n base points (§4.2, Fig. errors)."""
        tot, cnt = 0.0, 0
        for s0 in range(0, n, 2_000_000):
            x = sdev.points_cuda(mix, sd.STREAM_BASE, s0, min(2_000_000, n - s0), device=dev)
            tot += float(ix.encoding_error(x).double().sum())
            cnt += x.shape[0]
        return tot / cnt

    k, nq = 100, w.n_query
    out = {"workload": w.name, "n_base": w.n_base, "T": w.T, "M": w.M, "n_query": nq, "k": k, "dtype": "f32",
           "data": "synthetic", "l2": "flushed between timed runs (512 MB write)",
           "timing": "CUDA events, median of 5 after 3 warm-up (1 after 1 for the O(D) scorers)"}
    nn = exact_nn_gpu(q[:1000], w, mix, dev)
    if name == "c3":
        L, S = 30_000, 1000
        ix, out["build_s"] = build("global")
        loc16 = bpq.Index.train(learn, w.T, w.M, variant="local", iters=w.kmeans_iters)
        del learn
        eg, el = enc_error(ix), enc_error(loc16)
        del loc16
        out["encoding_error_16B"] = {"global": eg, "local": el, "reduction": 1.0 - el / eg,
                                     "points": "first 10M base points", "paper": "about 30 % lower (Fig. errors)"}
        ms32 = timed(lambda: ix.search(q, L, k, "fbpq"))
        a_ids, a_d = ix.search(q, L, k, "fbpq")
        A = a_ids.cpu().numpy()
        out.update({"L": L, "shortlist": S,
                    "lut": "int8 (per-query step) and fp16 (power-of-two step), offsets per sub-quantizer",
                    "fbpq_f32": {"qps": nq / (ms32 / 1e3), "ms": ms32, "recall": recall_of(a_ids[:1000], nn)}})
        for prec, key in (("int8", "shortlist_i8"), ("fp16", "shortlist_f16")):
            ms = timed(lambda: ix.search_shortlist(q, L, k, shortlist=S, precision=prec))
            b_ids, b_d = ix.search_shortlist(q, L, k, shortlist=S, precision=prec)
            B = b_ids.cpu().numpy()
            overlap = np.mean([len(np.intersect1d(A[n], B[n])) / k for n in range(nq)])
            same = a_ids == b_ids
            out[key] = {"qps": nq / (ms / 1e3), "ms": ms, "recall": recall_of(b_ids[:1000], nn),
                        "identical_lists": float(same.all(1).float().mean()), "mean_top100_overlap": float(overlap),
                        "max_abs_dist_diff_same_rank": float((a_d - b_d).abs()[same].max()) if same.any() else None}
        out["index"] = {"device_bytes": int(ix.info().device_bytes)}
    elif name == "c4":
        Ls = np.round(10.0 ** np.random.default_rng(7).uniform(3.0, 5.0, nq)).astype(np.int64)
        out.update({"L": "round(10^U(3,5)) per query, seed 7", "L_mean": float(Ls.mean())})
        ixl, out["build_local_s"] = build("local")
        el = enc_error(ixl)
        for scorer in ("hbpq", "hbpq_recon"):
            full = scorer == "hbpq"
            ms = timed(lambda: ixl.search(q, Ls, k, scorer), reps=5 if full else 1, warm=3 if full else 1)
            ids, _ = ixl.search(q, Ls, k, scorer)
            out[scorer] = {"qps": nq / (ms / 1e3), "ms": ms, "recall": recall_of(ids[:1000], nn)}
        out["batching_hbpq"] = batching_block(ixl, q, Ls, k, "hbpq", reps=10)
        out["index_local"] = {"device_bytes": int(ixl.info().device_bytes)}
        del ixl
        ixg, out["build_global_s"] = build("global")
        del learn
        eg = enc_error(ixg)
        out["encoding_error_8B"] = {"global": eg, "local": el, "reduction": 1.0 - el / eg,
                                    "points": "first 10M base points", "paper": "about 30 % lower (Fig. errors)"}
        for scorer in ("fbpq", "recon"):
            full = scorer == "fbpq"
            ms = timed(lambda: ixg.search(q, Ls, k, scorer), reps=5 if full else 1, warm=3 if full else 1)
            ids, _ = ixg.search(q, Ls, k, scorer)
            out[scorer] = {"qps": nq / (ms / 1e3), "ms": ms, "recall": recall_of(ids[:1000], nn)}
        out["hbpq_over_fbpq_time"] = out["hbpq"]["ms"] / out["fbpq"]["ms"]
        out["batching_fbpq"] = batching_block(ixg, q, Ls, k, "fbpq", reps=10)
        out["index_global"] = {"device_bytes": int(ixg.info().device_bytes)}
    elif name == "opq":
        # OMulti-D-OADC (the OPQ variant of the paper's experiments) next to the plain index
        ixp, _ = build("global")
        ixo, out["build_opq_s"] = build("global", opq=True)
        del learn
        out["encoding_error"] = {"plain": enc_error(ixp), "opq": enc_error(ixo), "points": "first 10M base points"}
        for L in w.L:
            row = {}
            for tag, ixx in (("plain", ixp), ("opq", ixo)):
                ms = timed(lambda: ixx.search(q, L, k, "fbpq"), reps=3, warm=2)
                ids, _ = ixx.search(q[:1000], L, k, "fbpq")
                row[tag] = {"qps": nq / (ms / 1e3), "ms": ms, "recall": recall_of(ids, nn)}
            out[f"L{L}"] = row
        out["index"] = {"device_bytes_opq": int(ixo.info().device_bytes)}
    elif name == "gist":
        # the paper's GIST50M rows (Table FBPQ): FBPQ vs reconstruction at D = 384, 8-byte codes
        ix, out["build_s"] = build("global")
        del learn
        out["index"] = {"device_bytes": int(ix.info().device_bytes)}
        out["dim"] = w.dim
        for L in w.L:
            row = {}
            for scorer in ("fbpq", "fbpq_tables", "recon"):
                full = scorer != "recon"
                ms = timed(lambda: ix.search(q, L, k, scorer), reps=3 if full else 1, warm=2 if full else 1)
                row[scorer] = {"qps": nq / (ms / 1e3), "ms": ms}
            ids, _ = ix.search(q[:1000], L, k, "fbpq")
            ids_r, _ = ix.search(q[:1000], L, k, "recon")
            row["recall_fbpq"] = recall_of(ids, nn)
            row["recall_recon"] = recall_of(ids_r, nn)
            row["speedup_fbpq_over_recon"] = row["recon"]["ms"] / row["fbpq"]["ms"]
            out[f"L{L}"] = row
        out["paper_cpu_speedup"] = {"L10000": 10.5, "L30000": 13.2, "L100000": 14.6}
    else:
        ix, out["build_s"] = build("global")
        del learn
        info = ix.info()
        cross_bytes = info.n_points * 4
        out["index"] = {"device_bytes": int(info.device_bytes), "n_points": int(info.n_points),
                        "per_point_cross_bytes": int(cross_bytes),
                        "device_bytes_without_per_point_cross": int(info.device_bytes - cross_bytes)}
        out["batch"] = {}
        for L in w.L:
            for scorer in ("fbpq", "fbpq_tables"):
                ms = timed(lambda: ix.search(q, L, k, scorer), reps=3, warm=2)
                out["batch"][f"{scorer}_L{L}"] = {"qps": nq / (ms / 1e3), "ms": ms}
        ids, _ = ix.search(q[:1000], 10_000, k, "fbpq")
        out["recall_L10000"] = recall_of(ids, nn)
        out["serve"] = serve_block(ix, w, mix, k, serve_seconds, n_max=200_000)
    return out


def run_config(args):
    """--workload c3 | c4 | c5: one configuration block as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(config_block(args.workload, args.serve_seconds)), flush=True)


def recall(ix, queries, w, mix, L, k, dev, n_gt=1000):
    """Recall@1/10/100 of the search against exact nearest neighbours (brute force
    in FP32 with TF32 off: every partial sum is an integer below 2^24, so exact)."""
    import torch

    from synthdata import device as sdev
    import synthdata as sd
    q = queries[:n_gt]
    qn = (q * q).sum(1, keepdim=True)
    best = torch.full((n_gt,), float("inf"), device=dev)
    arg = torch.zeros(n_gt, dtype=torch.int64, device=dev)
    chunk = 1_000_000
    for s in range(0, w.n_base, chunk):
        x = sdev.points_cuda(mix, sd.STREAM_BASE, s, min(chunk, w.n_base - s), device=dev)
        d = qn - 2.0 * (q @ x.T) + (x * x).sum(1)[None, :]
        m, a = d.min(1)
        upd = m < best
        best = torch.where(upd, m, best)
        arg = torch.where(upd, a + s, arg)
    out = {}
    for scorer in ("fbpq", "recon"):
        ids, _ = ix.search(q, L, k, scorer)
        hit = (ids.long() == arg[:, None])
        out[scorer] = {f"R@{R}": float(hit[:, :R].any(1).float().mean()) for R in (1, 10, 100)}
    out["n_queries"] = n_gt
    out["L"] = L
    return out


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, rank 0 only."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args)
    per_step = 2
    total = per_step * (args.steps + args.warmup)
    res = run_oracle(w, args.L, args.k, seconds=1e9, nq_max=total, multi=False)
    times = res["times"][per_step * args.warmup:]
    seconds = sum(times)
    value = len(times) / seconds
    sample = oracle_sample_text(w, args.L, per_step) + f" per step ({args.steps} timed steps, {args.warmup} warm-up)"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * seconds / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": w.name, "n_base": w.n_base, "dim": w.dim, "T": w.T, "M": w.M, "L": args.L,
                      "k": args.k, "scorer": "fbpq"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "sift10m":
        run_config(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
