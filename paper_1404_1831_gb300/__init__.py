"""Python binding of libbpq, the GB300 (sm_103a) bilayer product-quantization search library.

Argument marshalling only: every step of training, encoding, traversal and
scoring runs in the CUDA kernels behind the C ABI of ``include/bpq.h``.  PyTorch
provides device memory and streams.  There is no CPU fallback: if
``libbpq.so`` is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

BPQ_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "EIO", -4: "ECORRUPT", -5: "ETIMEOUT", -6: "ECUDA", -7: "ECAPACITY",
          -8: "ESTATE"}
VARIANT_GLOBAL, VARIANT_LOCAL = 0, 1
SCORERS = {"fbpq": 0, "recon": 1, "hbpq": 2, "fbpq_tables": 3, "hbpq_recon": 4}
LUT_PRECISIONS = {"int8": 1, "fp16": 2}


class BpqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int32), ("T", ctypes.c_int32), ("M", ctypes.c_int32), ("ksub", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("kmeans_iters", ctypes.c_int32), ("opq", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_pending", ctypes.c_int64), ("n_nonempty", ctypes.c_int64),
                ("max_cell", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("params", Params)]


class Arrays(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("C1", "C2", "R", "Q", "S", "X1", "X2", "offsets", "codes", "ids",
                                                "cross")]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("k", ctypes.c_int32), ("scorer", ctypes.c_int32),
                ("group_by_budget", ctypes.c_int32), ("max_batch", ctypes.c_int64), ("L_max", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t)]


class ServerStats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("queries", ctypes.c_int64), ("max_in_flight", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("slot_workspace_bytes", ctypes.c_int64)]


CELL_DTYPE = np.dtype([("cell", "<u4"), ("begin", "<u4"), ("count", "<u4"), ("key", "<f4")])

# Every entry point of include/bpq.h, with its ctypes signature.
_P = ctypes.c_void_p
_SIGS = {
    "bpq_last_error": (ctypes.c_char_p, []),
    "bpq_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Params), _P, _P, _P, _P, _P, ctypes.c_int]),
    "bpq_train_load": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Params), _P, ctypes.c_int64,
                                      ctypes.c_char_p, ctypes.c_int, _P]),
    "bpq_encode": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    "bpq_add": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "bpq_reconstruction_error": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "bpq_finalize": (ctypes.c_int, [_P, _P]),
    "bpq_set_global_counts": (ctypes.c_int, [_P, _P]),
    "bpq_query_tables": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "bpq_search_workspace_size": (ctypes.c_size_t, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                                    ctypes.c_int32]),
    "bpq_traverse": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P,
                                    ctypes.c_size_t, _P]),
    "bpq_search": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P,
                                  _P, _P, ctypes.c_size_t, _P]),
    "bpq_search_status": (ctypes.c_int, [_P, _P, _P]),
    "bpq_set_hbpq_table_budget": (ctypes.c_int, [_P, ctypes.c_double]),
    "bpq_set_scan_work_size": (ctypes.c_int, [_P, ctypes.c_int32]),
    "bpq_set_rotations": (ctypes.c_int, [_P, _P, _P, _P]),
    "bpq_get_rotations": (ctypes.c_int, [_P, _P, _P, _P]),
    "bpq_autotune": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P,
                                    _P, _P, _P]),
    "bpq_graph_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, ctypes.c_int64, _P, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "bpq_graph_set_budgets": (ctypes.c_int, [_P, _P]),
    "bpq_graph_launch": (ctypes.c_int, [_P, _P]),
    "bpq_graph_free": (None, [_P]),
    "bpq_search_shortlist_workspace_size": (ctypes.c_size_t, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]),
    "bpq_search_shortlist": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t, _P]),
    "bpq_scan": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                _P, _P, _P, _P]),
    "bpq_search_host": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       _P, _P, _P]),
    "bpq_search_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_int32, _P, _P, _P, _P]),
    "bpq_get_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "bpq_get_arrays": (ctypes.c_int, [_P, ctypes.POINTER(Arrays)]),
    "bpq_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "bpq_free": (None, [_P]),
    "bpq_server_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.POINTER(ServerConfig)]),
    "bpq_server_submit": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
    "bpq_server_progress": (ctypes.c_int, [_P, ctypes.c_int32]),
    "bpq_server_take": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    "bpq_server_run_trace": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "bpq_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "bpq_server_free": (None, [_P]),
}

_LIB = None


def library_path():
    return os.path.join(HERE, "libbpq.so")


def lib():
    """The loaded libbpq.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        so = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(so, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = so
    return _LIB


def _check(rc):
    if rc != BPQ_OK:
        raise BpqError(rc, lib().bpq_last_error().decode())


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _L_array(L, nq):
    L = np.asarray(L, dtype=np.int64)
    if L.ndim == 0:
        return np.ascontiguousarray(L.reshape(1)), 0
    if L.shape != (nq,):
        raise ValueError("L must be a scalar or have one value per query")
    return np.ascontiguousarray(L), 1


class _CudaView:
    """Wraps a raw device pointer for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


class Index:
    """An inverted multi-index with PQ-coded displacements on one GPU."""

    def __init__(self, handle, device=0):
        self._h = handle
        self.device = device
        self._ws = None

    # -- construction ---------------------------------------------------------
    @staticmethod
    def _params(D, T, M, variant, iters, opq=False):
        return Params(D=D, T=T, M=M, ksub=256, variant=variant, kmeans_iters=iters, opq=1 if opq else 0)

    @classmethod
    def create(cls, C1, C2, R, Q=None, S=None, device=0, rotations=None):
        """Index from host codebooks: C1, C2 (T, D/2); R (M, 256, D/M); Q, S (T, M/2, 256, D/M) for HBPQ;
        rotations = (R0 (D, D), R1, R2 (D/2, D/2)) for an OPQ index (codebooks in the rotated spaces)."""
        C1 = np.ascontiguousarray(C1, dtype=np.float32)
        C2 = np.ascontiguousarray(C2, dtype=np.float32)
        R = np.ascontiguousarray(R, dtype=np.float32)
        T, h = C1.shape
        M = R.shape[0]
        variant = VARIANT_LOCAL if Q is not None else VARIANT_GLOBAL
        p = cls._params(2 * h, T, M, variant, 0, opq=rotations is not None)
        qs = [np.ascontiguousarray(a, dtype=np.float32) if a is not None else None for a in (Q, S)]
        h_out = ctypes.c_void_p()
        _check(lib().bpq_create(ctypes.byref(h_out), ctypes.byref(p), C1.ctypes.data, C2.ctypes.data,
                                R.ctypes.data, qs[0].ctypes.data if qs[0] is not None else None,
                                qs[1].ctypes.data if qs[1] is not None else None, device))
        ix = cls(h_out, device)
        if rotations is not None:
            rs = [np.ascontiguousarray(r, dtype=np.float64) for r in rotations]
            _check(lib().bpq_set_rotations(ix._h, rs[0].ctypes.data, rs[1].ctypes.data, rs[2].ctypes.data))
        return ix

    @classmethod
    def train(cls, learn, T, M, variant="global", iters=10, stream=None, opq=False):
        """Train codebooks on the GPU from an (n, D) float32 CUDA tensor of integer-valued vectors
        (opq: with OPQ rotations learned first)."""
        import torch
        assert learn.is_cuda and learn.dtype == torch.float32 and learn.is_contiguous()
        v = VARIANT_LOCAL if variant == "local" else VARIANT_GLOBAL
        p = cls._params(learn.shape[1], T, M, v, iters, opq=opq)
        h_out = ctypes.c_void_p()
        _check(lib().bpq_train_load(ctypes.byref(h_out), ctypes.byref(p), _ptr(learn), learn.shape[0], None,
                                    learn.device.index or 0, _stream(stream)))
        return cls(h_out, learn.device.index or 0)

    @classmethod
    def load(cls, path, device=0):
        h_out = ctypes.c_void_p()
        _check(lib().bpq_train_load(ctypes.byref(h_out), None, None, 0, str(path).encode(), device, None))
        return cls(h_out, device)

    def save(self, path):
        _check(lib().bpq_save(self._h, str(path).encode()))

    def close(self):
        if self._h:
            lib().bpq_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- building -------------------------------------------------------------
    def encode(self, x, stream=None):
        import torch
        n = x.shape[0]
        cells = torch.empty(n, dtype=torch.int32, device=x.device)
        codes = torch.empty((n, self.params.M), dtype=torch.uint8, device=x.device)
        _check(lib().bpq_encode(self._h, _ptr(x), n, _ptr(cells), _ptr(codes), _stream(stream)))
        return cells, codes

    def add(self, x, ids=None, stream=None):
        _check(lib().bpq_add(self._h, _ptr(x), x.shape[0], _ptr(ids), _stream(stream)))

    def encoding_error(self, x, stream=None):
        """Squared encoding error ||x - xhat||^2 of every row of x (bpq_encode, then
        bpq_reconstruction_error): float32 (n,)."""
        import torch
        cells, codes = self.encode(x, stream)
        err = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _check(lib().bpq_reconstruction_error(self._h, _ptr(x), x.shape[0], _ptr(cells), _ptr(codes), _ptr(err),
                                              _stream(stream)))
        return err

    def finalize(self, stream=None):
        _check(lib().bpq_finalize(self._h, _stream(stream)))

    def cell_counts(self):
        """Points per cell (i*T + j) of this index's lists: int64 numpy (T*T,)."""
        import numpy as np
        off = self.arrays()["offsets"].cpu().numpy().view(np.uint32).astype(np.int64)
        return np.diff(off)

    def set_global_counts(self, counts):
        """Make this index a point shard: the whole index's per-cell counts (int64, T*T)
        drive the traversal, the shard's own lists the scan (bpq_set_global_counts).
        None clears it."""
        import numpy as np
        if counts is None:
            _check(lib().bpq_set_global_counts(self._h, None))
            return
        c = np.ascontiguousarray(counts, dtype=np.int64)
        p = self.params
        if c.shape != (p.T * p.T,):
            raise ValueError(f"counts must have shape ({p.T * p.T},)")
        _check(lib().bpq_set_global_counts(self._h, c.ctypes.data))

    # -- introspection --------------------------------------------------------
    def info(self):
        out = Info()
        _check(lib().bpq_get_info(self._h, ctypes.byref(out)))
        return out

    @property
    def params(self):
        return self.info().params

    def arrays(self):
        """Copies of the index arrays as CUDA tensors."""
        import torch
        a = Arrays()
        _check(lib().bpq_get_arrays(self._h, ctypes.byref(a)))
        inf = self.info()
        p = inf.params
        h, s, m2, n = p.D // 2, p.D // p.M, p.M // 2, inf.n_points
        shapes = {"C1": ((p.T, h), "<f4"), "C2": ((p.T, h), "<f4"), "R": ((p.M, 256, s), "<f4"),
                  "Q": ((p.T, m2, 256, s), "<f4"), "S": ((p.T, m2, 256, s), "<f4"),
                  "X1": ((p.T, m2, 256), "<f4"), "X2": ((p.T, m2, 256), "<f4"),
                  "offsets": ((p.T * p.T + 1,), "<u4"), "codes": ((n, p.M), "|u1"), "ids": ((n,), "<i4"),
                  "cross": ((n,), "<f4")}
        out = {}
        dev = torch.device("cuda", self.device)
        for name, (shape, ts) in shapes.items():
            ptr = getattr(a, name)
            if not ptr or 0 in shape:
                out[name] = None
                continue
            if ts == "<u4":  # torch has no uint32 copies everywhere: view as int32
                ts = "<i4"
            out[name] = torch.as_tensor(_CudaView(ptr, shape, ts), device=dev).clone()
        return out

    # -- queries --------------------------------------------------------------
    def workspace(self, nq, L_max, k, scorer="fbpq", stream=None):
        import torch
        need = lib().bpq_search_workspace_size(self._h, nq, int(L_max), k, SCORERS[scorer])
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=torch.device("cuda", self.device))
        return self._ws

    def query_tables(self, q, lut=True, stream=None):
        import torch
        p = self.params
        nq = q.shape[0]
        d1 = torch.empty((nq, p.T), dtype=torch.float32, device=q.device)
        d2 = torch.empty((nq, p.T), dtype=torch.float32, device=q.device)
        lt = torch.empty((nq, p.M, 256), dtype=torch.float32, device=q.device) if lut else None
        _check(lib().bpq_query_tables(self._h, _ptr(q), nq, _ptr(d1), _ptr(d2), _ptr(lt), _stream(stream)))
        return d1, d2, lt

    def traverse(self, q, L, cap, stream=None):
        """Visited non-empty cells per query: (cells int32 (nq, cap, 4) raw bpq_cell, ncells, npoints)."""
        import torch
        nq = q.shape[0]
        Ls, stride = _L_array(L, nq)
        cells = torch.empty((nq, cap, 4), dtype=torch.int32, device=q.device)
        ncells = torch.empty(nq, dtype=torch.int32, device=q.device)
        npoints = torch.empty(nq, dtype=torch.int64, device=q.device)
        ws = self.workspace(nq, int(Ls.max()), 1)
        _check(lib().bpq_traverse(self._h, _ptr(q), nq, Ls.ctypes.data, stride, cap, _ptr(cells), _ptr(ncells),
                                  _ptr(npoints), _ptr(ws), ws.numel(), _stream(stream)))
        return cells, ncells, npoints

    def search(self, q, L, k, scorer="fbpq", stream=None, workspace=None, out=None):
        import torch
        nq = q.shape[0]
        Ls, stride = _L_array(L, nq)
        if out is None:
            ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
            dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        else:
            ids, dists = out
        ws = workspace if workspace is not None else self.workspace(nq, int(Ls.max()), k, scorer)
        _check(lib().bpq_search(self._h, _ptr(q), nq, Ls.ctypes.data, stride, k, SCORERS[scorer], _ptr(ids),
                                _ptr(dists), _ptr(ws), ws.numel(), _stream(stream)))
        return ids, dists

    def scan(self, q, lut, cells, ncells, k, scorer="fbpq", stream=None, out=None):
        """Scan + top-k on traversal output (cells from traverse())."""
        import torch
        nq, cap = cells.shape[0], cells.shape[1]
        if out is None:
            ids = torch.empty((nq, k), dtype=torch.int32, device=cells.device)
            dists = torch.empty((nq, k), dtype=torch.float32, device=cells.device)
        else:
            ids, dists = out
        if getattr(self, "_counter", None) is None:
            self._counter = torch.zeros(1, dtype=torch.int32, device=cells.device)
        _check(lib().bpq_scan(self._h, _ptr(q), nq, _ptr(lut), _ptr(cells), _ptr(ncells), cap, k, SCORERS[scorer],
                              _ptr(ids), _ptr(dists), _ptr(self._counter), _stream(stream)))
        return ids, dists

    def search_shortlist(self, q, L, k, shortlist=1000, precision="int8", stream=None, workspace=None):
        """bpq_search_shortlist: int8- or FP16-table scan to a shortlist, exact FBPQ re-score, top k."""
        import torch
        nq = q.shape[0]
        Ls, stride = _L_array(L, nq)
        ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        if workspace is None:
            need = lib().bpq_search_shortlist_workspace_size(self._h, nq, int(Ls.max()), shortlist)
            if self._ws is None or self._ws.numel() < need:
                self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=torch.device("cuda", self.device))
            workspace = self._ws
        _check(lib().bpq_search_shortlist(self._h, _ptr(q), nq, Ls.ctypes.data, stride, k, shortlist,
                                          LUT_PRECISIONS[precision], _ptr(ids), _ptr(dists), _ptr(workspace),
                                          workspace.numel(), _stream(stream)))
        return ids, dists

    def search_noalloc(self, q, L, k, scorer="fbpq", stream=None, status=None):
        """bpq_search_noalloc: the search with the library's built-in scratch array
        instead of a workspace, for callers that must not allocate device memory.
        Raises BpqError with the return code on failure (e.g. ECAPACITY for a
        batch larger than the built-in scratch)."""
        import torch
        nq = q.shape[0]
        Ls, stride = _L_array(L, nq)
        ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        rc = lib().bpq_search_noalloc(self._h, _ptr(q), nq, Ls.ctypes.data, stride, k, SCORERS[scorer], _ptr(ids),
                                      _ptr(dists), _ptr(status), _stream(stream))
        if rc != BPQ_OK:
            raise BpqError(rc, "bpq_search_noalloc failed")
        return ids, dists

    def set_hbpq_table_budget(self, slots_per_query):
        """Table slots reserved per query by the HBPQ table form (0 = automatic)."""
        _check(lib().bpq_set_hbpq_table_budget(self._h, float(slots_per_query)))

    def rotations(self):
        """(R0, R1, R2) of an OPQ index as FP64 host arrays."""
        p = self.params
        R0 = np.empty((p.D, p.D))
        R1 = np.empty((p.D // 2, p.D // 2))
        R2 = np.empty((p.D // 2, p.D // 2))
        _check(lib().bpq_get_rotations(self._h, R0.ctypes.data, R1.ctypes.data, R2.ctypes.data))
        return R0, R1, R2

    def set_scan_work_size(self, candidates_per_item):
        """0: one CTA per query; W > 0: persistent work-queue scan with items of about W candidates."""
        _check(lib().bpq_set_scan_work_size(self._h, int(candidates_per_item)))

    def autotune(self, q, L, k, scorer="fbpq", stream=None):
        """bpq_autotune on this batch: returns the chosen work-item size (0 = one CTA per query)."""
        import torch
        nq = q.shape[0]
        Ls, stride = _L_array(L, nq)
        ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        chosen = ctypes.c_int32()
        _check(lib().bpq_autotune(self._h, _ptr(q), nq, Ls.ctypes.data, stride, k, SCORERS[scorer], _ptr(ids),
                                  _ptr(dists), _stream(stream), ctypes.byref(chosen)))
        return chosen.value

    def graph(self, q, L, k, scorer="fbpq"):
        """A SearchGraph: this batch shape captured once, replayed by launch()."""
        return SearchGraph(self, q, L, k, scorer)

    def search_status(self, workspace=None, stream=None):
        ws = workspace if workspace is not None else self._ws
        _check(lib().bpq_search_status(self._h, _ptr(ws), _stream(stream)))

    def search_host(self, q, L, k, scorer="fbpq", stream=None):
        """Host numpy queries in, host numpy (ids, dists) out; copies are inside the call."""
        q = np.ascontiguousarray(q, dtype=np.float32)
        nq = q.shape[0]
        Ls, stride = _L_array(L, nq)
        ids = np.empty((nq, k), dtype=np.int32)
        dists = np.empty((nq, k), dtype=np.float32)
        _check(lib().bpq_search_host(self._h, q.ctypes.data, nq, Ls.ctypes.data, stride, k, SCORERS[scorer],
                                     ids.ctypes.data, dists.ctypes.data, _stream(stream)))
        return ids, dists


class SearchGraph:
    """bpq_graph_*: static device buffers q (nq, D), ids / dists (nq, k); write new
    queries into .q (and new budgets with set_budgets) before launch()."""

    def __init__(self, index, q, L, k, scorer="fbpq"):
        import torch
        self.index = index
        self.q = q
        nq = q.shape[0]
        self.ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        self.dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        Ls, stride = _L_array(L, nq)
        h = ctypes.c_void_p()
        _check(lib().bpq_graph_create(ctypes.byref(h), index._h, _ptr(q), nq, Ls.ctypes.data, stride, k,
                                      SCORERS[scorer], _ptr(self.ids), _ptr(self.dists)))
        self._h = h

    def set_budgets(self, L):
        Ls = np.ascontiguousarray(L, dtype=np.int64)
        _check(lib().bpq_graph_set_budgets(self._h, Ls.ctypes.data))

    def launch(self, stream=None):
        _check(lib().bpq_graph_launch(self._h, _stream(stream)))
        return self.ids, self.dists

    def close(self):
        if getattr(self, "_h", None):
            lib().bpq_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def header_symbols():
    """Function names declared in include/bpq.h."""
    import re
    hdr = open(os.path.join(os.path.dirname(HERE), "include", "bpq.h")).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(bpq_\w+)\s*\(", hdr, flags=re.M)))
