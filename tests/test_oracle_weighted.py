"""Pins of the weighted-graph oracle (NEXT f3: Section 3.3 after Algorithm 2,
weights uniform in [1, 100] as in Section 5).

Two independent forms of the weighted ADS are in the oracle: Algorithm 1 in
Dijkstra order (the definition) and the paper's Algorithm 2 in BFS-order
supersteps with CleanUp.  They are pinned against each other, against a
brute-force ADS from Floyd-Warshall distances, and against the unweighted
oracle when every length is 1.  The radius, the MIS on weighted balls and
the weighted assignment are pinned against the brute-force definitions on
the same distance table."""
import math

import numpy as np
import pytest

import brute
import flsynth
import oracle


def _graphs():
    out = {}
    out["path"] = brute.csr_from_edges(9, [(i, i + 1) for i in range(8)])
    out["star"] = brute.csr_from_edges(8, [(0, i) for i in range(1, 8)])
    out["cycle"] = brute.csr_from_edges(11, [(i, (i + 1) % 11) for i in range(11)])
    out["mixed"] = brute.csr_from_edges(12, [(0, 1), (1, 2), (2, 3), (3, 0), (1, 4), (4, 5), (5, 6), (6, 4),
                                             (7, 8), (9, 10), (10, 11), (9, 11), (2, 9)])
    w = flsynth.small_er(26, 3.0, 17)
    out["er26"] = (w.rowp, w.cols)
    return out


GRAPHS = _graphs()


def _weighted(name, seed=5, lo=1, hi=100):
    rowp, cols = GRAPHS[name]
    return rowp, cols, flsynth.edge_weights(rowp, cols, seed, lo, hi)


def _ads_rows(A, n):
    """Per vertex: list of (distance, [ids in rank order], counted, weight)."""
    rows = []
    for v in range(n):
        g0, g1 = A["gofs"][v], A["gofs"][v + 1]
        e = A["eofs"][v]
        groups = []
        for gi in range(g0, g1):
            c = int(A["gcnt"][gi])
            groups.append((int(A["ghop"][gi]), [int(x) for x in A["eid"][e:e + c]], int(A["gcounted"][gi]),
                           float(A["gwt"][gi])))
            e += c
        rows.append(groups)
    return rows


def test_edge_weights_symmetric_and_in_range():
    rowp, cols = GRAPHS["er26"]
    w = flsynth.edge_weights(rowp, cols, 9)
    assert w.min() >= 1 and w.max() <= 100
    pos = {}
    for v in range(len(rowp) - 1):
        for e in range(rowp[v], rowp[v + 1]):
            pos[(v, int(cols[e]))] = int(w[e])
    assert all(pos[(u, v)] == x for (v, u), x in pos.items())
    # the full range is used on a larger graph (uniform draws)
    big = flsynth.small_er(3000, 8.0, 3)
    wb = flsynth.edge_weights(big.rowp, big.cols, 1)
    assert wb.min() == 1 and wb.max() == 100 and abs(wb.mean() - 50.5) < 1.5


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [2, 4, 16])
def test_weighted_ads_matches_brute_force(name, k):
    """The definitional build against the ADS recomputed from Floyd-Warshall
    distances: entries, distances, counted prefixes and HIP weights."""
    rowp, cols, w = _weighted(name)
    n = len(rowp) - 1
    D = brute.apsp_weighted(rowp, cols, w)
    rk = oracle.ranks(3, n)
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(k, 3)
    got = _ads_rows(g.ads(), n)
    want = brute.ads_by_definition(D, rk, k)
    for v in range(n):
        assert [h for h, *_ in got[v]] == [h for h, _ in want[v]]
        for (h, ids, counted, wt), (wh, ents) in zip(got[v], want[v]):
            assert ids == [e[1] for e in ents]
            flags = [e[2] for e in ents]
            assert counted == sum(flags) and all(flags[:counted])
            for e in ents:
                if e[2]:
                    assert e[3] == wt
    # hops: the largest distance of an ADS entry
    assert g.hops == max(h for v in range(n) for h, _ in want[v])


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [2, 4, 16])
def test_algorithm2_with_cleanup_equals_dijkstra_order(name, k):
    """The paper's BFS-order supersteps with CleanUp reach the same ADS
    (entries and distances) as Algorithm 1 in Dijkstra order."""
    rowp, cols, w = _weighted(name)
    n = len(rowp) - 1
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(k, 7)
    A = g.ads()
    R = g.wads_rounds(k, 7)
    D = brute.apsp_weighted(rowp, cols, w)
    for v in range(n):
        ids_def = [int(x) for x in A["eid"][A["eofs"][v]:A["eofs"][v + 1]]]
        ids_rnd = [int(x) for x in R["eid"][R["eofs"][v]:R["eofs"][v + 1]]]
        assert ids_def == ids_rnd
        dd = [int(x) for x in R["edist"][R["eofs"][v]:R["eofs"][v + 1]]]
        assert dd == [int(D[v, u]) for u in ids_rnd]


def test_cleanup_runs_where_bfs_order_is_not_distance_order():
    """A heavy direct edge and a light two-hop path: BFS order delivers the
    far copy first, so CleanUp must remove entries that a closer copy later
    invalidates, and the supersteps still end at the definition."""
    # vertices 0..5: 0-5 heavy (100), 0-1-2-3-4-5 light (1 each); plus a fan
    edges = [(0, 5), (0, 1), (1, 2), (2, 3), (3, 4), (4, 5)] + [(5, 6 + i) for i in range(6)]
    rowp, cols = brute.csr_from_edges(12, edges)
    w = np.ones(len(cols), np.int32)
    for v in range(12):
        for e in range(rowp[v], rowp[v + 1]):
            if {v, int(cols[e])} == {0, 5}:
                w[e] = 100
    k = 2
    cleaned_any = False
    for seed in range(1, 40):
        g = oracle.Graph(rowp, cols)
        g.set_weights(w)
        g.build_sketches_weighted(k, seed)
        A = g.ads()
        R = g.wads_rounds(k, seed)
        for v in range(12):
            assert list(A["eid"][A["eofs"][v]:A["eofs"][v + 1]]) == list(R["eid"][R["eofs"][v]:R["eofs"][v + 1]])
        cleaned_any |= R["cleaned"] > 0
    assert cleaned_any


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_unit_lengths_reduce_to_the_unweighted_build(name):
    """Every length 1: the weighted ADS is the hop ADS entry for entry,
    weight for weight, and the radii agree bit for bit."""
    rowp, cols = GRAPHS[name]
    n = len(rowp) - 1
    for k in (2, 4, 16):
        a = oracle.Graph(rowp, cols)
        a.build_sketches(k, 4)
        b = oracle.Graph(rowp, cols)
        b.set_weights(np.ones(len(cols), np.int32))
        b.build_sketches_weighted(k, 4)
        A, B = a.ads(), b.ads()
        for key in ("gofs", "eofs", "ghop", "gcnt", "gcounted", "eid"):
            assert np.array_equal(A[key], B[key]), key
        assert np.array_equal(A["gwt"].view(np.uint64), B["gwt"].view(np.uint64))
        cost = flsynth.loguniform(n, 8, 0.5, 30.0)
        client = flsynth.bernoulli(n, 9, 0.7)
        assert np.array_equal(a.radii(cost, client).view(np.uint64), b.radii(cost, client).view(np.uint64))


def test_hip_estimates_exact_when_the_graph_has_at_most_k_vertices():
    """n <= k: every weight is 1, so the estimated number of clients within
    distance d of v is the exact count (Floyd-Warshall)."""
    rowp, cols, w = _weighted("er26", seed=11)
    n = len(rowp) - 1
    D = brute.apsp_weighted(rowp, cols, w)
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(32, 2)
    A = g.ads()
    assert np.all(A["gwt"] == 1.0)
    client = flsynth.bernoulli(n, 4, 0.6)
    for v in range(n):
        e = A["eofs"][v]
        est = {}
        for gi in range(A["gofs"][v], A["gofs"][v + 1]):
            c = int(A["gcnt"][gi])
            est[int(A["ghop"][gi])] = sum(int(client[x]) for x in A["eid"][e:e + int(A["gcounted"][gi])])
            e += c
        for d in sorted(set(int(x) for x in D[v] if x >= 0)):
            exact = sum(int(client[u]) for u in range(n) if 0 <= D[v, u] <= d)
            assert sum(c for h, c in est.items() if h <= d) == exact


def test_radius_exact_with_exact_counts():
    """n <= k: r_f solves sum_c max(0, r - d(c, f)) = c(f) over clients at
    their weighted distances (rational arithmetic)."""
    rowp, cols, w = _weighted("er26", seed=12, lo=1, hi=9)
    n = len(rowp) - 1
    D = brute.apsp_weighted(rowp, cols, w)
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(32, 3)
    client = flsynth.bernoulli(n, 5, 0.7)
    cost = flsynth.loguniform(n, 6, 0.5, 60.0)
    r = g.radii(cost, client)
    for f in range(n):
        dists = [int(D[f, c]) for c in range(n) if client[c] and D[f, c] >= 0]
        want = brute.exact_radius(dists, cost[f])
        if want is None:
            assert not math.isfinite(r[f])
        else:
            assert abs(r[f] - float(want)) <= 1e-12 * max(1.0, float(want))


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_mis_on_weighted_balls_is_the_lexicographically_first(name):
    """Selection with Ball(f) = clients within distance floor(r_f): the
    lexicographically-first MIS of H-bar built from Floyd-Warshall."""
    rowp, cols, w = _weighted(name, seed=21, lo=1, hi=12)
    n = len(rowp) - 1
    D = brute.apsp_weighted(rowp, cols, w)
    for seed in (1, 2, 3):
        g = oracle.Graph(rowp, cols)
        g.set_weights(w)
        g.build_sketches_weighted(4, seed)
        client = flsynth.bernoulli(n, 30 + seed, 0.6)
        fac = flsynth.bernoulli(n, 40 + seed, 0.6)
        cost = flsynth.loguniform(n, 50 + seed, 1.0, 80.0, fac)
        r = g.radii(cost, client)
        op, nopen = g.open_facilities_weighted(r, client, seed)
        cand, balls, adj = brute.conflict_graph(D, r, client)
        S = brute.lfmis(cand, adj, key=lambda f: (r[f], oracle.priority(seed, f)))
        assert set(np.flatnonzero(op)) == S and nopen == len(S)


@pytest.mark.parametrize("hi", [1, 3])
def test_mis_chain_of_rounds_on_a_path(hi):
    """A path whose costs grow along it, every vertex a client: each ball
    overlaps the next one, so the lexicographically-first MIS is a long chain
    of dependent decisions (the case where a parallel greedy needs many
    rounds); against brute force on Floyd-Warshall distances."""
    n = 80
    rowp, cols = brute.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    w = flsynth.edge_weights(rowp, cols, 21, 1, hi)
    D = brute.apsp_weighted(rowp, cols, w)
    cost = np.linspace(2.0, 8.0, n) * hi
    client = np.ones(n, np.uint8)
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(4, 0)
    r = g.radii(cost, client)
    op, nopen = g.open_facilities_weighted(r, client, 0)
    cand, balls, adj = brute.conflict_graph(D, r, client)
    S = brute.lfmis(cand, adj, key=lambda f: (r[f], oracle.priority(0, f)))
    assert set(np.flatnonzero(op)) == S and nopen == len(S)
    assert 1 < len(S) < n


def test_components_without_facilities_and_huge_costs():
    """Small components, some without a facility (their clients stay
    unassigned: -1, -1), opening costs up to 1e9 so that balls cover whole
    components: selection and assignment against brute force."""
    wl = flsynth.small_er(40, 1.2, 87)
    n = wl.n
    w = flsynth.edge_weights(wl.rowp, wl.cols, 15)
    D = brute.apsp_weighted(wl.rowp, wl.cols, w)
    fac = flsynth.bernoulli(n, 40, 0.3)
    cost = flsynth.loguniform(n, 41, 1.0, 1.0e9, fac)
    client = flsynth.bernoulli(n, 42, 0.5)
    g = oracle.Graph(wl.rowp, wl.cols)
    g.set_weights(w)
    g.build_sketches_weighted(8, 9)
    r = g.radii(cost, client)
    op, nopen = g.open_facilities_weighted(r, client, 9)
    cand, balls, adj = brute.conflict_graph(D, r, client)
    S = brute.lfmis(cand, adj, key=lambda f: (r[f], oracle.priority(9, f)))
    assert set(np.flatnonzero(op)) == S and nopen == len(S)
    a, d = g.assign_weighted(op)
    wa, wd = brute.nearest_assignment(D, S)
    assert np.array_equal(a, wa) and np.array_equal(d, wd)
    assert (d < 0).any() and (d > 0).any()
    assert max(np.floor(r[f]) for f in cand) > 1.0e5  # balls far wider than any distance


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_weighted_assignment_is_the_nearest_open_facility(name):
    rowp, cols, w = _weighted(name, seed=23)
    n = len(rowp) - 1
    D = brute.apsp_weighted(rowp, cols, w)
    op = np.zeros(n, np.uint8)
    op[[0, n // 2, n - 1]] = 1
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    a, d = g.assign_weighted(op)
    wa, wd = brute.nearest_assignment(D, set(np.flatnonzero(op)))
    assert np.array_equal(a, wa) and np.array_equal(d, wd)


def test_solve_weighted_end_to_end():
    """The whole weighted path: the objective recomputed from the open set
    and Floyd-Warshall distances."""
    rowp, cols, w = _weighted("er26", seed=31)
    n = len(rowp) - 1
    D = brute.apsp_weighted(rowp, cols, w)
    client = flsynth.bernoulli(n, 61, 0.7)
    fac = flsynth.bernoulli(n, 62, 0.5)
    cost = flsynth.loguniform(n, 63, 5.0, 200.0, fac)
    out = oracle.solve_weighted(rowp, cols, w, 4, 1, cost, client)
    S = set(np.flatnonzero(out["open"]))
    _, wd = brute.nearest_assignment(D, S)
    served = [c for c in range(n) if client[c] and wd[c] >= 0]
    obj = sum(cost[f] for f in sorted(S)) + float(sum(int(wd[c]) for c in served))
    assert abs(out["objective"] - obj) <= 1e-9 * abs(obj)
    assert out["n_unserved"] == sum(1 for c in range(n) if client[c] and wd[c] < 0)


def test_bad_weights_rejected():
    rowp, cols = GRAPHS["path"]
    g = oracle.Graph(rowp, cols)
    with pytest.raises(ValueError):
        g.set_weights(np.zeros(len(cols), np.int32))
