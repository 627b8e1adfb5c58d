"""Device-side generation of the synthdata points (same bytes as synthdata.points).

Loads synthdata/libsynth.so (built by __graft_entry__.build()) and writes points
straight into torch CUDA tensors, so large workloads never cross the PCIe bus.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import Mixture, mix64_int

_LIB = None
_TABLES = {}


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth.so")
        if not os.path.exists(path):
            raise RuntimeError("synthdata/libsynth.so is missing; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        lib.synth_points.restype = ctypes.c_int
        lib.synth_points.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                             ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _LIB = lib
    return _LIB


def _tables(mix: Mixture, device):
    import torch
    key = (mix.seed, mix.n_comp, mix.dim, str(device))
    if key not in _TABLES:
        _TABLES[key] = (
            torch.as_tensor(mix.mu.astype(np.int32), device=device),
            torch.as_tensor(mix.sigma.astype(np.int32), device=device),
            torch.as_tensor(mix.cum.astype(np.uint64).view(np.int64), device=device),
            torch.as_tensor(np.ascontiguousarray(mix.B.astype(np.int32)), device=device),
        )
    return _TABLES[key]


def points_cuda(mix: Mixture, stream: int, start: int, count: int, dtype="float32", device="cuda", out=None):
    """Points start .. start+count-1 of a stream as a (count, dim) CUDA tensor."""
    import torch
    mu, sigma, cum, B = _tables(mix, device)
    if out is None:
        out = torch.empty((count, mix.dim), dtype=torch.float32 if dtype == "float32" else torch.uint8,
                          device=device)
    f = out.data_ptr() if out.dtype == torch.float32 else None
    u = out.data_ptr() if out.dtype == torch.uint8 else None
    rc = _lib().synth_points(mu.data_ptr(), sigma.data_ptr(), cum.data_ptr(), B.data_ptr(), mix.n_comp, mix.dim,
                             mix64_int(mix.seed), stream, start, count, f, u,
                             torch.cuda.current_stream(out.device).cuda_stream)
    if rc != 0:
        raise RuntimeError(f"synth_points failed with CUDA error {rc}")
    return out
