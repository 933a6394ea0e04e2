"""C-ABI library: builds, loads, exports every declared symbol; host-side checks.

These run without a GPU: argument validation in the entry points happens
before any CUDA call.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1503_03635_gb300 as fl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fl.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fl_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("fl_graph_create", "fl_build_sketches", "fl_compute_radii", "fl_open_facilities",
                 "fl_assign_clients", "fl_objective"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    path = fl.load().__getattribute__("_name")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fl_[a-z_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert set(declared_symbols()) == set(fl.EXPORTS)


def test_library_is_built_for_sm_103a():
    """Every object is compiled and linked with exactly one -gencode, for sm_103a."""
    from paper_1503_03635_gb300 import build

    assert build.ARCH == "-gencode=arch=compute_103a,code=sm_103a"
    assert build.ARCH in build.NVCC_FLAGS
    assert sum(f.startswith("-gencode") or f.startswith("-arch") for f in build.NVCC_FLAGS) == 1


def test_binding_checks_tensor_dtypes():
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        fl.Graph(torch.zeros(3, dtype=torch.int32), torch.zeros(2, dtype=torch.int32))
    with pytest.raises(TypeError):
        fl.Graph(torch.zeros(3, dtype=torch.int64), torch.zeros(2, dtype=torch.int64))


def test_status_strings_and_last_error():
    lib = fl.load()
    assert lib.fl_status_str(0) == b"ok"
    assert lib.fl_status_str(fl.FL_EINVAL) == b"invalid argument"
    assert lib.fl_status_str(fl.FL_ETIMEOUT) == b"iteration limit reached"
    assert lib.fl_status_str(99) == b"unknown status"


def test_graph_create_rejects_bad_arguments_on_host():
    lib = fl.load()
    h = ctypes.c_void_p()
    rowp = np.zeros(2, np.int64)
    cols = np.zeros(0, np.int32)
    # n < 1
    rc = lib.fl_graph_create(0, rowp.ctypes.data_as(ctypes.c_void_p), cols.ctypes.data_as(ctypes.c_void_p),
                             0, fl.FL_MEM_HOST, None, ctypes.byref(h))
    assert rc == fl.FL_EINVAL and not h.value
    buf = ctypes.create_string_buffer(256)
    assert lib.fl_last_error(buf, 256) == fl.FL_EINVAL
    assert b"n must be" in buf.value
    # bad memory kind
    rc = lib.fl_graph_create(1, rowp.ctypes.data_as(ctypes.c_void_p), cols.ctypes.data_as(ctypes.c_void_p),
                             0, 7, None, ctypes.byref(h))
    assert rc == fl.FL_EINVAL
    # null output pointer
    assert lib.fl_graph_create(1, None, None, 0, 0, None, None) == fl.FL_EINVAL


def test_null_handles_are_rejected():
    lib = fl.load()
    assert lib.fl_build_sketches(None, 16, 1) == fl.FL_EINVAL
    assert lib.fl_sketch_stats(None, None, None, None, None) == fl.FL_EINVAL
    assert lib.fl_compute_radii(None, None, None, 0, None) == fl.FL_EINVAL
    assert lib.fl_open_facilities(None, None, None, 0) == fl.FL_EINVAL
    assert lib.fl_assign_clients(None, None, None, 0) == fl.FL_EINVAL
    assert lib.fl_objective(None, None, None, None) == fl.FL_EINVAL
    assert lib.fl_graph_destroy(None) == fl.FL_OK
    assert lib.fl_solve_destroy(None) == fl.FL_OK
    h = ctypes.c_void_p()
    assert lib.fl_solve_create(None, ctypes.byref(h)) == fl.FL_EINVAL


def test_binding_rejects_wrong_dtypes():
    with pytest.raises(TypeError):
        fl.Graph(np.zeros(3, np.int32), np.zeros(2, np.int32))


def test_oracle_is_not_imported_by_the_product():
    """The product package never imports, loads or links the oracle, and the
    oracle never imports the product."""
    pkg = os.path.join(ROOT, "paper_1503_03635_gb300")
    bad = re.compile(r"^\s*(import|from)\s+oracle\b|floracle|fl_oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                assert not bad.search(open(os.path.join(dirpath, f)).read()), f
    bad2 = re.compile(r"^\s*(import|from)\s+paper_1503_03635_gb300\b|libflgpu|fl_internal", re.M)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            assert not bad2.search(open(os.path.join(ROOT, "oracle", f)).read()), f


def test_schedule_struct_and_null_handles():
    lib = fl.load()
    assert ctypes.sizeof(fl.Schedule) == 24
    sc = fl.Schedule(0, 16, 8, 16, 0, 0)
    assert lib.fl_set_schedule(None, ctypes.byref(sc)) == fl.FL_EINVAL
    assert lib.fl_get_schedule(None, ctypes.byref(sc)) == fl.FL_EINVAL
    assert lib.fl_batch_set_schedule(None, ctypes.byref(sc)) == fl.FL_EINVAL
    assert lib.fl_autotune(None, 16, 1, None, None, 0, 4, None, None, None) == fl.FL_EINVAL
    assert lib.fl_eps_stats(None, None, None, None, None, None) == fl.FL_EINVAL
    assert lib.fl_open_facilities_eps(None, 0.1, None, None, 0, None, None, None, None) == fl.FL_EINVAL
    assert lib.fl_autotune_forget() == fl.FL_OK
