"""Build the CUDA libraries in-tree with nvcc (sm_103a only).

  paper_1404_1831_gb300/libbpq.so   the search library (C ABI of include/bpq.h)
  synthdata/libsynth.so             the device-side input generator

Translation units compile in parallel; objects go to paper_1404_1831_gb300/_build/.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]
BPQ_SOURCES = ["bpq_api.cu", "bpq_tables.cu", "bpq_traverse.cu", "bpq_scan.cu", "bpq_build.cu", "bpq_noalloc.cu",
               "bpq_hbpq.cu", "bpq_serve.cu", "bpq_graph.cu",
               "bpq_opq.cu"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _needs(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, obj, deps):
    if not _needs(obj, [src] + deps):
        return obj
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def build(verbose=False):
    csrc = os.path.join(HERE, "csrc")
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    headers = [os.path.join(csrc, "bpq_internal.cuh"), os.path.join(ROOT, "include", "bpq.h")]
    jobs = [(os.path.join(csrc, s), os.path.join(bdir, s.replace(".cu", ".o")), headers) for s in BPQ_SOURCES]
    synth_src = os.path.join(ROOT, "synthdata", "csrc", "synth.cu")
    synth_obj = os.path.join(bdir, "synth.o")
    jobs.append((synth_src, synth_obj, []))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    outs = [(os.path.join(HERE, "libbpq.so"), objs[:-1]), (os.path.join(ROOT, "synthdata", "libsynth.so"), objs[-1:])]
    for so, parts in outs:
        if _needs(so, parts):
            cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", *parts, "-o", so]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed for {so}:\n{r.stderr}")
        if verbose:
            print("built", so)
    return [o for o, _ in outs]


if __name__ == "__main__":
    build(verbose=True)
