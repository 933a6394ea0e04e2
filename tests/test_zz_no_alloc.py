"""The allocation-free assignment entry point (for callers that cannot let the
library allocate device memory) against the regular assignment.

Kept in a file that pytest collects last.  Both calls in a row must match the
assignment of fl_assign_clients on the same graph and open set exactly.
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
