"""GPU parity of the weighted-graph path (NEXT f3: Section 3.3 after
Algorithm 2; weights uniform in [1, 100] as in Section 5) through the C ABI,
against the oracle's weighted ADS, selection and assignment.

Bit-exact: sketches, ADS groups (distance, entry count, counted prefix),
entry ids and HIP weights, the largest distance, the open set (balls by
weighted distance), assignments and distances, the distance sum; radii and
the objective within 1e-9 relative (radii in practice bit-identical: the
same operation order).  The oracle's ADS is pinned to the paper's
Algorithm 2 with CleanUp and to Floyd-Warshall brute force, its selection to
the lexicographically-first MIS by brute force and its assignment to
all-pairs distances (tests/test_oracle_weighted.py), so these cases also show
that the Dijkstra-order build on the GPU ends where CleanUp does."""
import numpy as np
import pytest

import brute
import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def _compare(rowp, cols, w, k, seed, cost, client):
    n = len(rowp) - 1
    og = oracle.Graph(rowp, cols)
    og.set_weights(w)
    og.build_sketches_weighted(k, seed)
    A = og.ads(ranks=False)
    S_o, cnt_o = og.sketch()
    g = fl.Graph(rowp, cols, lengths=w)
    g.build_sketches(k, seed)
    st = g.stats()
    assert st["hops"] == og.hops and st["edge_merges"] == 0
    S, cnt = g.export_sketches()
    assert np.array_equal(cnt, cnt_o) and np.array_equal(S, S_o)
    B = g.export_ads()
    for key in ("gofs", "eofs", "ghop", "gcnt", "gcounted", "eid"):
        assert np.array_equal(A[key], B[key]), key
    assert np.array_equal(A["gwt"].view(np.uint64), B["gwt"].view(np.uint64))
    s = fl.Solve(g)
    r = s.compute_radii(cost, client)
    ro = og.radii(cost, client)
    fin = np.isfinite(ro)
    assert np.array_equal(np.isfinite(r), fin)
    assert np.all(np.abs(r[fin] - ro[fin]) <= RTOL * np.abs(ro[fin]))
    # selection and assignment by weighted distance
    op, nopen = s.open_facilities()
    op_o, nopen_o = og.open_facilities_weighted(ro, client, seed)
    assert nopen == nopen_o and np.array_equal(op, op_o)
    a, d = s.assign_clients()
    a_o, d_o = og.assign_weighted(op_o)
    assert np.array_equal(d, d_o) and np.array_equal(a, a_o)
    obj, ds, un = s.objective()
    obj_o, ds_o, un_o = oracle.objective(op_o, cost, client, d_o)
    assert ds == ds_o and un == un_o
    assert abs(obj - obj_o) <= RTOL * abs(obj_o)
    st["mis"] = s.stats()
    st["mis_log"] = s.mis_log()
    st["n_open"] = nopen
    s.close()
    g.close()
    og.close()
    return st


def _inputs(n, seed, fac_p=0.5, cli_p=0.7, lo=1.0, hi=400.0):
    fac = flsynth.bernoulli(n, seed, fac_p)
    return flsynth.loguniform(n, seed + 1, lo, hi, fac), flsynth.bernoulli(n, seed + 2, cli_p)


@pytest.mark.parametrize("kind", ["path", "star", "cycle", "two"])
@pytest.mark.parametrize("k", [2, 4, 16, 32])
def test_tiny_graphs(kind, k):
    if kind == "path":
        rowp, cols = brute.csr_from_edges(14, [(i, i + 1) for i in range(13)])
    elif kind == "star":
        rowp, cols = brute.csr_from_edges(11, [(0, i) for i in range(1, 11)])
    elif kind == "cycle":
        rowp, cols = brute.csr_from_edges(13, [(i, (i + 1) % 13) for i in range(13)])
    else:
        rowp, cols = brute.csr_from_edges(14, [(i, i + 1) for i in range(7)] + [(8 + i, 9 + i) for i in range(5)])
    n = len(rowp) - 1
    w = flsynth.edge_weights(rowp, cols, 3)
    cost, client = _inputs(n, 70)
    _compare(rowp, cols, w, k, 5, cost, client)


@pytest.mark.parametrize("k", [4, 16, 32])
def test_er_graph_full_weight_range(k):
    """Erdos-Renyi, 3000 vertices, lengths uniform in [1, 100]: many levels,
    rows of tens of entries, the cursor skipping across levels."""
    wl = flsynth.small_er(3000, 6.0, 81)
    w = flsynth.edge_weights(wl.rowp, wl.cols, 7)
    cost, client = _inputs(wl.n, 90)
    st = _compare(wl.rowp, wl.cols, w, k, 2, cost, client)
    assert st["hops"] > 100


@pytest.mark.parametrize("scale,k", [(11, 16), (13, 32)])
def test_rmat_with_hubs(scale, k):
    """R-MAT with hubs: warps merging candidates from thousands of edges,
    many duplicates of one rank arriving over different edges in one level."""
    rowp, cols = flsynth.rmat(scale, 16, 300 + scale)
    n = len(rowp) - 1
    w = flsynth.edge_weights(rowp, cols, 11)
    cost, client = _inputs(n, 95, fac_p=0.3, cli_p=0.5, lo=10.0, hi=1.0e4)
    _compare(rowp, cols, w, k, 1, cost, client)


def test_narrow_weights_many_ties():
    """Lengths in [1, 3]: many vertices at one distance (ties by rank) and
    consecutive levels."""
    wl = flsynth.small_er(2000, 5.0, 83)
    w = flsynth.edge_weights(wl.rowp, wl.cols, 9, 1, 3)
    cost, client = _inputs(wl.n, 97)
    _compare(wl.rowp, wl.cols, w, 16, 3, cost, client)


def test_unit_lengths_equal_the_unweighted_build():
    rowp, cols = flsynth.rmat(12, 16, 512)
    n = len(rowp) - 1
    a = fl.Graph(rowp, cols)
    a.build_sketches(16, 4)
    b = fl.Graph(rowp, cols, lengths=np.ones(len(cols), np.int32))
    b.build_sketches(16, 4)
    A, B = a.export_ads(), b.export_ads()
    for key in ("gofs", "eofs", "ghop", "gcnt", "gcounted", "eid"):
        assert np.array_equal(A[key], B[key]), key
    assert np.array_equal(A["gwt"].view(np.uint64), B["gwt"].view(np.uint64))
    assert a.stats()["hops"] == b.stats()["hops"]
    a.close()
    b.close()


def test_device_memory_inputs():
    torch = pytest.importorskip("torch")
    wl = flsynth.small_er(1500, 5.0, 85)
    w = flsynth.edge_weights(wl.rowp, wl.cols, 13)
    dev = torch.device("cuda:0")
    g = fl.Graph(torch.from_numpy(wl.rowp).to(dev), torch.from_numpy(wl.cols).to(dev),
                 lengths=torch.from_numpy(w).to(dev))
    g.build_sketches(16, 6)
    h = fl.Graph(wl.rowp, wl.cols, lengths=w)
    h.build_sketches(16, 6)
    A, B = g.export_ads(), h.export_ads()
    for key in A:
        assert np.array_equal(A[key], B[key]), key
    g.close()
    h.close()


@pytest.mark.parametrize("hi", [1, 3, 10])
def test_chain_of_greedy_rounds(hi):
    """A path whose costs grow along it: each facility's ball overlaps the
    next one's, so the greedy decides a few facilities per round (about 30
    rounds), each round's kill sweep deciding who drops out."""
    n = 240
    rowp, cols = brute.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    w = flsynth.edge_weights(rowp, cols, 21, 1, hi)
    cost = np.linspace(2.0, 8.0, n) * hi
    client = np.ones(n, np.uint8)
    st = _compare(rowp, cols, w, 4, 0, cost, client)
    assert st["mis"]["mis_rounds"] >= (20 if hi == 1 else 2)
    log = st["mis_log"]
    tot = log[log[:, 1] == 3]
    assert len(tot) == st["mis"]["mis_rounds"]
    # every candidate is decided in exactly one greedy round
    assert tot[:, 4].sum() == st["n_open"]
    assert np.all(np.diff(tot[:, 3]) < 0)  # the undecided set shrinks every round


def test_components_huge_radii_and_unserved_clients():
    """Many small components (some without a facility: unserved clients,
    assignment -1), costs up to 1e9 so that balls cover whole components and
    the largest ball radius is far above every distance: the sweeps skip the
    idle stretches between entry times."""
    wl = flsynth.small_er(600, 1.2, 87)
    w = flsynth.edge_weights(wl.rowp, wl.cols, 15)
    fac = flsynth.bernoulli(wl.n, 40, 0.15)
    cost = flsynth.loguniform(wl.n, 41, 1.0, 1.0e9, fac)
    client = flsynth.bernoulli(wl.n, 42, 0.5)
    _compare(wl.rowp, wl.cols, w, 8, 9, cost, client)


def test_dense_conflicts_many_facilities():
    """Erdos-Renyi with nearly every vertex a facility and a client, small
    costs and lengths in [1, 10]: overlapping balls in every round."""
    wl = flsynth.small_er(1200, 3.0, 89)
    w = flsynth.edge_weights(wl.rowp, wl.cols, 17, 1, 10)
    fac = flsynth.bernoulli(wl.n, 43, 0.9)
    cost = flsynth.loguniform(wl.n, 44, 1.0, 30.0, fac)
    client = flsynth.bernoulli(wl.n, 45, 0.9)
    st = _compare(wl.rowp, wl.cols, w, 16, 10, cost, client)
    log = st["mis_log"]
    tot = log[log[:, 1] == 3]
    assert tot[:, 4].sum() == st["n_open"]  # the rows count the facilities that joined


def test_unbuilt_calls_and_bad_lengths():
    rowp, cols = brute.csr_from_edges(10, [(i, i + 1) for i in range(9)])
    n = len(rowp) - 1
    w = flsynth.edge_weights(rowp, cols, 1)
    g = fl.Graph(rowp, cols, lengths=w)
    g.build_sketches(4, 1)
    s = fl.Solve(g)
    cost, client = _inputs(n, 50)
    s.compute_radii(cost, client)
    for call in (lambda: s.open_facilities_eps(0.1, cost, client), lambda: s.compute_radii_exact(cost, client)):
        with pytest.raises(fl.FLError) as e:
            call()
        assert e.value.status == fl.FL_ESTATE
    s.close()
    g.close()
    for bad in (0, -3, 70000):
        wb = w.copy()
        wb[len(wb) // 2] = bad
        with pytest.raises(fl.FLError) as e:
            fl.Graph(rowp, cols, lengths=wb)
        assert e.value.status == fl.FL_EINVAL
    # a length that differs between the two directions of an edge
    wb = w.copy()
    wb[0] = w[0] % 100 + 1
    with pytest.raises(fl.FLError) as e:
        fl.Graph(rowp, cols, lengths=wb)
    assert e.value.status == fl.FL_EINVAL
    with pytest.raises(ValueError):
        fl.Graph(rowp, cols, lengths=w[:-1])
