"""GPU parity of batches (fl_batch_*): every instance of a batch gives the
result of the plain fl_* sequence on that instance alone (bit-exact open
sets, assignments, distances, counts; objective within 1e-9 relative), and
equals the oracle's result for that instance (every instance of the union
batches, four instances of the replica batch)."""
import numpy as np
import pytest

import brute
import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def _plain(rowp, cols, k, seed, cost, client):
    return fl.solve(rowp, cols, k, seed, cost, client)


def _check_instance(res, lo, hi, i, want):
    assert np.array_equal(res["open"][lo:hi], want["open"]), i
    assert np.array_equal(res["assign"][lo:hi], want["assign"]), i
    assert np.array_equal(res["dist"][lo:hi], want["dist"]), i
    assert res["n_open"][i] == want["n_open"], i
    assert res["dist_sum"][i] == want["dist_sum"] and res["n_unserved"][i] == want["n_unserved"], i
    assert abs(res["objective"][i] - want["objective"]) <= RTOL * abs(want["objective"]), i


def _instances():
    """Graphs of uneven size: tiny graphs, small ER, an R-MAT with hubs, a
    graph without edges; random client subsets and costs."""
    out = []
    for name, (rowp, cols) in [("path", brute.csr_from_edges(12, [(i, i + 1) for i in range(11)])),
                               ("star", brute.csr_from_edges(9, [(0, i) for i in range(1, 9)]))]:
        out.append((rowp, cols))
    for j, (n, deg) in enumerate([(1000, 4.0), (3000, 9.0), (500, 14.0), (20000, 6.0)]):
        w = flsynth.small_er(n, deg, 300 + j)
        out.append((w.rowp, w.cols))
    out.append(flsynth.rmat(13, 16, 77))
    out.append((np.zeros(6, np.int64), np.zeros(0, np.int32)))
    return out


@pytest.mark.parametrize("k", [4, 32])
def test_union_batch_matches_plain_solves(k):
    graphs = _instances()
    costs, clients = [], []
    for i, (rowp, cols) in enumerate(graphs):
        n = len(rowp) - 1
        fac = flsynth.bernoulli(n, 900 + i, 0.6)
        costs.append(np.where(fac > 0, flsynth.loguniform(n, 910 + i, 2.0, 400.0), np.inf))
        clients.append(flsynth.bernoulli(n, 920 + i, 0.7))
    b = fl.Batch.union(graphs)
    assert b.n_inst == len(graphs)
    res = b.solve(k, 3, np.concatenate(costs), np.concatenate(clients))
    lo = 0
    for i, (rowp, cols) in enumerate(graphs):
        n = len(rowp) - 1
        want = _plain(rowp, cols, k, 3, costs[i], clients[i])
        _check_instance(res, lo, lo + n, i, want)
        # every instance of the batch against the oracle, too
        _check_instance(res, lo, lo + n, i, oracle.solve(rowp, cols, k, 3, costs[i], clients[i]))
        lo += n
    # a second solve on the same batch (new costs) is independent of the first
    costs2 = [np.where(np.isfinite(c), c * 1.7, np.inf) for c in costs]
    res2 = b.solve(k, 3, np.concatenate(costs2), np.concatenate(clients))
    lo = 0
    for i, (rowp, cols) in enumerate(graphs):
        n = len(rowp) - 1
        _check_instance(res2, lo, lo + n, i, _plain(rowp, cols, k, 3, costs2[i], clients[i]))
        lo += n
    b.close()


def test_replica_batch_matches_plain_solves_on_the_resident_graph():
    rowp, cols = flsynth.rmat(14, 16, 515)
    n = len(rowp) - 1
    k, seed = 16, 5
    g = fl.Graph(rowp, cols)
    g.build_sketches(k, seed)
    R = 6
    costs, clients = [], []
    for i in range(R):
        fac = flsynth.bernoulli(n, 1000 + i, 0.2 + 0.1 * i)
        c = np.full(n, float(flsynth.uniform(1, 1010 + i, 5.0, 500.0)[0]))
        costs.append(np.where(fac > 0, c, np.inf))
        clients.append(flsynth.bernoulli(n, 1020 + i, 0.05 + 0.15 * i))
    b = fl.Batch.replicas(g, R)
    assert (b.n_inst, b.n_total) == (R, R * n)
    res = b.solve(k, seed, np.concatenate(costs), np.concatenate(clients))
    for i in range(R):
        s = fl.Solve(g)
        s.compute_radii(costs[i], clients[i])
        op, no = s.open_facilities()
        a, d = s.assign_clients()
        obj, ds, un = s.objective()
        s.close()
        want = dict(open=op, assign=a, dist=d, n_open=no, objective=obj, dist_sum=ds, n_unserved=un)
        _check_instance(res, i * n, (i + 1) * n, i, want)
    # the first 2 instances alone (a prefix of the batch), then all again
    part = b.solve(k, seed, np.concatenate(costs[:2]), np.concatenate(clients[:2]), n_active=2)
    assert len(part["open"]) == 2 * n and len(part["objective"]) == 2
    for i in range(2):
        _check_instance(part, i * n, (i + 1) * n, i, {key: res[key][i * n:(i + 1) * n] if key in
                                                      ("open", "assign", "dist") else res[key][i]
                                                      for key in res})
    # four instances against the oracle's solve on the resident graph
    og = oracle.Graph(rowp, cols)
    og.build_sketches(k, seed)
    for i in (0, 2, 4, 5):
        r = og.radii(costs[i], clients[i])
        op, no = og.open_facilities(r, clients[i], seed)
        a, d = og.assign(op)
        obj, ds, un = oracle.objective(op, costs[i], clients[i], d)
        _check_instance(res, i * n, (i + 1) * n, i, dict(open=op, assign=a, dist=d, n_open=no, objective=obj,
                                                         dist_sum=ds, n_unserved=un))
    og.close()
    again = b.solve(k, seed, np.concatenate(costs), np.concatenate(clients))
    for key in ("open", "assign", "dist", "n_open", "dist_sum", "n_unserved"):
        assert np.array_equal(again[key], res[key])
    # the solve must use the resident graph's k and seed
    with pytest.raises(fl.FLError):
        b.solve(k, seed + 1, np.concatenate(costs), np.concatenate(clients))
    b.close()
    g.close()


def test_union_batch_rejects_edges_that_leave_their_graph():
    a = brute.csr_from_edges(4, [(0, 1), (2, 3)])
    bad_cols = a[1].copy()
    bad_cols[0] = 5  # a valid id of the union, but outside graph 0
    with pytest.raises(fl.FLError):
        fl.Batch.union([(a[0], bad_cols), brute.csr_from_edges(4, [(0, 1)])])
    bad_rowp = a[0].copy()
    bad_rowp[-1] += 1  # offsets do not end at nnz
    with pytest.raises(fl.FLError):
        fl.Batch.union([(bad_rowp, a[1]), brute.csr_from_edges(4, [(0, 1)])])
    starts_late = a[0].copy()
    starts_late[0] = 1  # offsets do not start at 0
    with pytest.raises(fl.FLError):
        fl.Batch.union([brute.csr_from_edges(4, [(0, 1)]), (starts_late, a[1])])
