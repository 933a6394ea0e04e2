"""Schedules change how the kernels lay out work, never the results: every
schedule gives bit-identical sketches, ADS, open sets, assignments and
objectives; the autotuner picks one, sets it, and caches it per graph
signature."""
import numpy as np
import pytest

import flsynth
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu

SCHEDULES = [
    dict(hop_group=32),
    dict(sparse_div=1),
    dict(sparse_div=1024),
    dict(dense_div=1, edge_div=1),       # rounds push unless the frontier is everything
    dict(dense_div=1024, edge_div=1024),  # rounds pull almost always
    dict(hop_group=32, sparse_div=64, dense_div=2, edge_div=4),
    dict(graph_bfs=1),                    # the assignment BFS as one CUDA graph
]


def _run(w, **sched):
    g = fl.Graph(w.rowp, w.cols)
    if sched:
        g.set_schedule(**sched)
    g.build_sketches(w.k, w.seed)
    S, cnt = g.export_sketches()
    ads = g.export_ads()
    s = fl.Solve(g)
    r = s.compute_radii(w.cost, w.client)
    op, no = s.open_facilities()
    a, d = s.assign_clients()
    obj = s.objective()
    s.close()
    g.close()
    return dict(S=S, cnt=cnt, ads=ads, r=r, open=op, n_open=no, assign=a, dist=d, obj=obj)


def _workloads():
    rowp, cols = flsynth.rmat(14, 16, 88)
    n = len(rowp) - 1
    cost = flsynth.loguniform(n, 5, 5.0, 500.0)
    rm = flsynth.from_csr("rmat14", rowp, cols, 16, 1, cost, flsynth.bernoulli(n, 6, 0.6))
    return [flsynth.config("er10k"), rm, flsynth.from_csr("rmat14k32", rowp, cols, 32, 3, cost, rm.client)]


@pytest.mark.parametrize("wi", [0, 1, 2])
def test_every_schedule_gives_identical_results(wi):
    w = _workloads()[wi]
    base = _run(w)
    for sched in SCHEDULES:
        got = _run(w, **sched)
        assert np.array_equal(got["S"], base["S"]) and np.array_equal(got["cnt"], base["cnt"]), sched
        for key in base["ads"]:
            a, b = got["ads"][key], base["ads"][key]
            if a.dtype == np.float64:
                a, b = a.view(np.uint64), b.view(np.uint64)
            assert np.array_equal(a, b), (sched, key)
        assert np.array_equal(got["r"].view(np.uint64), base["r"].view(np.uint64)), sched
        for key in ("open", "assign", "dist"):
            assert np.array_equal(got[key], base[key]), (sched, key)
        assert got["n_open"] == base["n_open"] and got["obj"] == base["obj"], sched


def test_bad_schedules_are_rejected():
    w = flsynth.config("er10k")
    g = fl.Graph(w.rowp, w.cols)
    for bad in (dict(hop_group=8), dict(sparse_div=0), dict(dense_div=2000), dict(edge_div=-1), dict(graph_bfs=2),
                dict(level_cap=-1)):
        with pytest.raises(fl.FLError):
            g.set_schedule(**bad)
    assert g.schedule == dict(hop_group=0, sparse_div=16, dense_div=8, edge_div=16, graph_bfs=0, level_cap=0)
    g.close()


def test_autotune_sets_a_schedule_and_caches_it():
    fl.autotune_forget()
    w = _workloads()[1]
    g = fl.Graph(w.rowp, w.cols)
    t = g.autotune(w.k, w.seed, w.cost, w.client, max_trials=6)
    assert g.schedule == t["schedule"] and t["ms_tuned"] <= t["ms_default"] * 1.0 + 1e-9
    # the graph is left built, and the tuned schedule gives the default results
    base = _run(w)
    s = fl.Solve(g)
    s.compute_radii(w.cost, w.client)
    op, _ = s.open_facilities()
    a, _ = s.assign_clients()
    assert np.array_equal(op, base["open"]) and np.array_equal(a, base["assign"])
    s.close()
    # a second graph of the same signature takes the cached choice
    g2 = fl.Graph(w.rowp, w.cols)
    t2 = g2.autotune(w.k, w.seed, w.cost, w.client, max_trials=6)
    assert t2 == t and g2.schedule == t["schedule"]
    g.close()
    g2.close()
    fl.autotune_forget()


def test_batch_schedule_gives_identical_results():
    rowp, cols = flsynth.rmat(12, 16, 515)
    n = len(rowp) - 1
    g = fl.Graph(rowp, cols)
    g.build_sketches(16, 5)
    cost = np.concatenate([np.full(n, 40.0), np.full(n, 90.0)])
    client = np.concatenate([flsynth.bernoulli(n, 7, 0.3), flsynth.bernoulli(n, 8, 0.6)])
    b = fl.Batch.replicas(g, 2)
    base = b.solve(16, 5, cost, client)
    b.set_schedule(dict(hop_group=0, sparse_div=16, dense_div=1024, edge_div=1024, graph_bfs=1, level_cap=0))
    got = b.solve(16, 5, cost, client)
    for key in ("open", "assign", "dist", "n_open", "dist_sum", "n_unserved"):
        assert np.array_equal(got[key], base[key]), key
    b.close()
    g.close()


@pytest.mark.parametrize("graph_bfs", [0, 1])
def test_bfs_level_cap_returns_etimeout(graph_bfs):
    """A BFS that needs more levels than the cap stops with FL_ETIMEOUT (the
    device-side loop of the graph form and the host-driven form alike); the
    context stays usable and the next solve with enough levels succeeds."""
    import brute

    rowp, cols = brute.csr_from_edges(40, [(i, i + 1) for i in range(39)])  # a path: 39 levels from vertex 0
    g = fl.Graph(rowp, cols)
    g.build_sketches(16, 1)
    cost = np.full(40, np.inf)
    cost[0] = 1.0
    client = np.ones(40, np.uint8)
    g.set_schedule(graph_bfs=graph_bfs, level_cap=5)
    s = fl.Solve(g)
    s.compute_radii(cost, client)
    s.open_facilities()
    with pytest.raises(fl.FLError) as e:
        s.assign_clients()
    assert e.value.status == fl.FL_ETIMEOUT
    g.set_schedule(level_cap=0)
    a, d = s.assign_clients()
    assert (a == 0).all() and np.array_equal(d, np.arange(40))
    s.close()
    g.close()
