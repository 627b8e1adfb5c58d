"""The C-ABI library loads and exports every entry point include/bpq.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1404_1831_gb300 as bpq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so():
    if not os.path.exists(bpq.library_path()):
        from paper_1404_1831_gb300 import _build
        _build.build()
    return ctypes.CDLL(bpq.library_path())


def test_header_declares_expected_entry_points():
    names = bpq.header_symbols()
    for n in ("bpq_train_load", "bpq_add", "bpq_encode", "bpq_finalize", "bpq_search", "bpq_traverse",
              "bpq_query_tables", "bpq_save", "bpq_free", "bpq_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(so):
    for name in bpq.header_symbols():
        assert hasattr(so, name), name
    assert set(bpq.header_symbols()) == set(bpq._SIGS)


def test_struct_layouts_match_header():
    hdr = open(os.path.join(ROOT, "include", "bpq.h")).read()
    params = re.search(r"typedef struct \{([^{}]*)\} bpq_params;", hdr, re.S).group(1)
    fields = re.findall(r"int32_t (\w+);", params)
    assert [f for f, _ in bpq.Params._fields_] == fields and ctypes.sizeof(bpq.Params) == 4 * len(fields)
    cfg = re.search(r"typedef struct \{([^{}]*)\} bpq_server_config;", hdr, re.S).group(1)
    assert [f for f, _ in bpq.ServerConfig._fields_] == re.findall(r"(?:int32_t|int64_t|size_t) (\w+);", cfg)
    assert bpq.CELL_DTYPE.itemsize == 16
    assert re.search(r"uint32_t cell;.*uint32_t begin;.*uint32_t count;.*float key;", hdr, re.S)


def test_cpu_calls_fail_cleanly_without_gpu(so):
    """Argument errors are reported as return codes, not crashes."""
    lib = bpq.lib()
    out = ctypes.c_void_p()
    rc = lib.bpq_create(ctypes.byref(out), None, None, None, None, None, None, 0)
    assert rc == -1 and out.value is None
    assert lib.bpq_last_error()
    assert lib.bpq_search_workspace_size(None, 10, 10, 10, 0) == 0
    p = bpq.Params(D=128, T=64, M=7, ksub=256, variant=0, kmeans_iters=1)
    assert lib.bpq_train_load(ctypes.byref(out), ctypes.byref(p), None, 0, None, 0, None) == -1
