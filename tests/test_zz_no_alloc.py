"""The allocation-free assignment entry point (for callers that cannot let the
library allocate device memory) against the regular assignment.

Kept in a file that pytest collects last.  Both calls in a row must match the
assignment of fl_assign_clients on the same graph and open set exactly.  The
Python wrapper checks types, lengths and devices before anything is launched;
the CPU tests below plant each mismatch and expect it to raise there.
"""
import ctypes

import numpy as np
import pytest

import flsynth
import paper_1503_03635_gb300 as fl


def test_noalloc_rejects_oversized_graph_on_host():
    lib = fl.load()
    rc = lib.fl_assign_nearest_noalloc((1 << 20) + 1, None, None, 0, None, None, None, None)
    assert rc == fl.FL_EINVAL
    buf = ctypes.create_string_buffer(256)
    lib.fl_last_error(buf, 256)
    assert b"fixed scratch" in buf.value


def _cpu_args(torch, n=5, nnz=6):
    rowp = torch.tensor([0, 2, 3, 4, 5, 6], dtype=torch.int64)[: n + 1]
    cols = torch.tensor([1, 2, 0, 0, 4, 3], dtype=torch.int32)[:nnz]
    op = torch.zeros(n, dtype=torch.uint8)
    a = torch.zeros(n, dtype=torch.int32)
    d = torch.zeros(n, dtype=torch.int32)
    return rowp, cols, op, a, d


@pytest.mark.parametrize("bad", ["rowp_i32", "cols_i64", "open_f32", "assign_i64", "open_short",
                                 "dist_long", "rowp_2d", "host_memory", "no_outputs", "numpy"])
def test_noalloc_wrapper_rejects_mismatches_before_launch(bad):
    torch = pytest.importorskip("torch")
    rowp, cols, op, a, d = _cpu_args(torch)
    if bad == "rowp_i32":
        rowp = rowp.to(torch.int32)
    elif bad == "cols_i64":
        cols = cols.to(torch.int64)
    elif bad == "open_f32":
        op = op.to(torch.float32)
    elif bad == "assign_i64":
        a = a.to(torch.int64)
    elif bad == "open_short":
        op = op[:-1]
    elif bad == "dist_long":
        d = torch.zeros(6, dtype=torch.int32)
    elif bad == "rowp_2d":
        rowp = rowp.reshape(2, 3)
    elif bad == "no_outputs":
        a = d = None
    elif bad == "numpy":
        cols = cols.numpy()
    # every case fails in the wrapper; "host_memory" is the well-typed call,
    # which fails because the tensors are not in device memory
    with pytest.raises((TypeError, ValueError)):
        fl.assign_nearest_noalloc(rowp, cols, op, a, d)


def _regular_assignment(w):
    g = fl.Graph(w.rowp, w.cols)
    g.build_sketches(w.k, w.seed)
    s = fl.Solve(g)
    s.compute_radii(w.cost, w.client)
    op, nopen = s.open_facilities()
    a, d = s.assign_clients()
    s.close()
    g.close()
    assert nopen > 0
    return op, a, d


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["er10k", "rmat20"])
def test_noalloc_matches_regular_assignment_twice(name):
    torch = pytest.importorskip("torch")
    w = flsynth.config(name)  # rmat20 has exactly the 2^20-vertex limit
    op, a_ref, d_ref = _regular_assignment(w)
    dev = torch.device("cuda:0")
    rowp = torch.from_numpy(w.rowp).to(dev)
    cols = torch.from_numpy(w.cols).to(dev)
    open_d = torch.from_numpy(op).to(dev)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        a = torch.full((w.n,), -7, dtype=torch.int32, device=dev)
        d = torch.full((w.n,), -7, dtype=torch.int32, device=dev)
        fl.assign_nearest_noalloc(rowp, cols, open_d, a, d, stream=stream)
        assert np.array_equal(a.cpu().numpy(), a_ref)
        assert np.array_equal(d.cpu().numpy(), d_ref)


@pytest.mark.gpu
def test_noalloc_invalid_csr_and_unreachable_component():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    # offsets that decrease (every read stays inside the arrays) -> FL_EINVAL
    rowp = torch.tensor([0, 3, 1, 4, 4], dtype=torch.int64, device=dev)
    cols = torch.tensor([1, 2, 3, 0], dtype=torch.int32, device=dev)
    op = torch.tensor([1, 0, 0, 0], dtype=torch.uint8, device=dev)
    a = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(fl.FLError) as e:
        fl.assign_nearest_noalloc(rowp, cols, op, a, None, stream=stream)
    assert e.value.status == fl.FL_EINVAL
    # a column outside [0, n) -> FL_EINVAL
    rowp = torch.tensor([0, 1, 2, 3, 4], dtype=torch.int64, device=dev)
    cols = torch.tensor([1, 0, 9, 2], dtype=torch.int32, device=dev)
    with pytest.raises(fl.FLError) as e:
        fl.assign_nearest_noalloc(rowp, cols, op, a, None, stream=stream)
    assert e.value.status == fl.FL_EINVAL
    # two components {0,1,2} (path, facility 0 open) and {3,4} (no facility):
    # the second one's vertices get -1 / -1, twice in a row
    rowp = torch.tensor([0, 1, 3, 4, 5, 6], dtype=torch.int64, device=dev)
    cols = torch.tensor([1, 0, 2, 1, 4, 3], dtype=torch.int32, device=dev)
    op = torch.tensor([1, 0, 0, 0, 0], dtype=torch.uint8, device=dev)
    for _ in range(2):
        a = torch.full((5,), 7, dtype=torch.int32, device=dev)
        d = torch.full((5,), 7, dtype=torch.int32, device=dev)
        fl.assign_nearest_noalloc(rowp, cols, op, a, d, stream=stream)
        assert a.cpu().tolist() == [0, 0, 0, -1, -1]
        assert d.cpu().tolist() == [0, 1, 2, -1, -1]
