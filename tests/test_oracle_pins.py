"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

Each test compares the oracle with something other than itself: published
generator outputs, brute-force definitions on tiny graphs (tests/brute.py),
closed forms, statistical unbiasedness, and structural invariants.
"""
import math
import os

import numpy as np
import pytest

import brute
import flsynth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- graphs

def path_graph(n):
    return brute.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])


def star_graph(leaves):
    return brute.csr_from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)])


def cycle_graph(n):
    return brute.csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def complete_graph(n):
    return brute.csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def two_components_and_isolated():
    # path 0-1-2-3, triangle 4-5-6, isolated 7, edge 8-9
    e = [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (4, 6), (8, 9)]
    return brute.csr_from_edges(10, e)


def small_er(n, avg, seed):
    return flsynth.er(n, int(n * avg / 2), seed)


TINY = {
    "path9": path_graph(9),
    "star7": star_graph(7),
    "cycle11": cycle_graph(11),
    "k6": complete_graph(6),
    "mixed": two_components_and_isolated(),
    "er40": small_er(40, 2.5, 5),
    "er60": small_er(60, 4.0, 6),
    "er30dense": small_er(30, 8.0, 9),
}


# ---------------------------------------------------------------- ranks

def test_splitmix64_published_vectors():
    """Rank generator = published SplitMix64 outputs (Algorithm 1's r(u))."""
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert rows
    for row in rows:
        state = int(row[0], 0)
        want = [int(x, 0) for x in row[1:]]
        assert oracle.splitmix64_outputs(state, len(want)) == want


def test_rank_is_generator_stream_and_injective():
    """r(v) is the (v+1)-th output from the seed; pi uses a second stream."""
    seed = 1
    outs = oracle.splitmix64_outputs(seed, 50)
    assert [oracle.rank(seed, v) for v in range(50)] == outs
    rk = oracle.ranks(seed, 5000)
    assert len(np.unique(rk)) == 5000
    first = oracle.splitmix64_outputs(seed, 1)[0]
    assert [oracle.priority(seed, f) for f in range(20)] == oracle.splitmix64_outputs(first, 20)


# ---------------------------------------------------------------- sketches

@pytest.mark.parametrize("name", sorted(TINY))
@pytest.mark.parametrize("k", [2, 4, 16])
def test_sketch_equals_bottom_k_of_component(name, k):
    """S at the fixed point = bottom-k ranks of the connected component."""
    rowp, cols = TINY[name]
    D = brute.apsp(rowp, cols)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(k, 3)
    S, cnt = g.sketch()
    rk = oracle.ranks(3, g.n)
    for v in range(g.n):
        want = brute.bottom_k([int(rk[w]) for w in range(g.n) if D[v, w] >= 0], k)
        assert cnt[v] == len(want)
        assert [int(x) for x in S[v, :cnt[v]]] == want
        assert all(int(x) == 2 ** 64 - 1 for x in S[v, cnt[v]:])


@pytest.mark.parametrize("name", sorted(TINY))
@pytest.mark.parametrize("k", [2, 3, 4, 16])
def test_ads_and_hip_weights_by_definition(name, k):
    """ADS entries, hops, counted flags and HIP weights equal the definition
    evaluated on all-pairs BFS balls (Section 3.3; HIP per Cohen 2014)."""
    rowp, cols = TINY[name]
    D = brute.apsp(rowp, cols)
    seed = 11
    rk = oracle.ranks(seed, len(rowp) - 1)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(k, seed)
    A = g.ads()
    want = brute.ads_by_definition(D, rk, k)
    for v in range(g.n):
        g0, g1 = A["gofs"][v], A["gofs"][v + 1]
        got_groups = []
        for gi in range(g0, g1):
            e0 = A["eofs"][v] + sum(A["gcnt"][g0:gi])
            ids = A["eid"][e0:e0 + A["gcnt"][gi]]
            rks = A["erank"][e0:e0 + A["gcnt"][gi]]
            got_groups.append((int(A["ghop"][gi]), [int(x) for x in rks], [int(x) for x in ids],
                               int(A["gcounted"][gi]), float(A["gwt"][gi])))
        assert [h for h, *_ in got_groups] == [h for h, _ in want[v]]
        for (h, rks, ids, counted, wt), (wh, went) in zip(got_groups, want[v]):
            assert rks == [e[0] for e in went]
            assert ids == [e[1] for e in went]
            flags = [e[2] for e in went]
            # counted entries come first (they are the smallest ranks)
            assert counted == sum(flags) and all(flags[:counted])
            for e in went:
                if e[2]:
                    assert e[3] == wt  # bit-exact: same IEEE division


@pytest.mark.parametrize("name", sorted(TINY))
def test_hop_count_and_edge_merges(name):
    """H* = last hop where some S_h changes; edge-merges = sum over processed
    hops of deg(u) for u whose sketch changed at the previous hop."""
    rowp, cols = TINY[name]
    k = 4
    D = brute.apsp(rowp, cols)
    rk = oracle.ranks(2, len(rowp) - 1)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(k, 2)
    n = g.n
    deg = np.diff(rowp)
    prev = [brute.sketch_at(D, rk, k, v, 0) for v in range(n)]
    changed_prev = [True] * n          # hop 0: every vertex is new
    merges, last = 0, 0
    h = 1
    while True:
        cur = [brute.sketch_at(D, rk, k, v, h) for v in range(n)]
        for v in range(n):
            merges += sum(1 for u in cols[rowp[v]:rowp[v + 1]] if changed_prev[u])
        changed = [cur[v] != prev[v] for v in range(n)]
        if not any(changed):
            break
        last = h
        prev, changed_prev = cur, changed
        h += 1
    assert g.hops == last
    assert g.edge_merges == merges


@pytest.mark.parametrize("name", ["er60", "mixed", "star7", "er30dense"])
def test_algorithm1_single_vertex_matches_propagation(name):
    """Algorithm 1 (sequential, per vertex) and hop-synchronous Algorithm 2
    build the same ADS for unweighted graphs (Section 3.3)."""
    rowp, cols = TINY[name]
    k = 4
    g = oracle.Graph(rowp, cols)
    g.build_sketches(k, 5)
    A = g.ads()
    for v in range(g.n):
        one = g.vertex_ads(k, 5, v)
        e0, e1 = A["eofs"][v], A["eofs"][v + 1]
        g0, g1 = A["gofs"][v], A["gofs"][v + 1]
        assert list(one["eid"]) == list(A["eid"][e0:e1])
        assert list(one["ghop"]) == list(A["ghop"][g0:g1])
        assert list(one["gcounted"]) == list(A["gcounted"][g0:g1])
        assert list(one["gwt"]) == list(A["gwt"][g0:g1])


def test_ads_size_bound():
    """|ADS(v)| <= k per distance, and at most one group per distance."""
    rowp, cols = flsynth.rmat(10, 8, 77)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(8, 1)
    A = g.ads()
    assert (A["gcnt"] <= 8).all() and (A["gcnt"] >= 1).all()
    for v in range(0, g.n, 7):
        hops = A["ghop"][A["gofs"][v]:A["gofs"][v + 1]]
        assert (np.diff(hops) > 0).all()


# ---------------------------------------------------------------- HIP

@pytest.mark.parametrize("name", ["path9", "star7", "k6", "mixed"])
def test_hip_exact_when_balls_are_small(name):
    """With every ball smaller than k all weights are 1 and the estimate is
    the exact (predicated) count."""
    rowp, cols = TINY[name]
    n = len(rowp) - 1
    k = 16
    D = brute.apsp(rowp, cols)
    client = (np.arange(n) % 3 != 1).astype(np.uint8)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(k, 4)
    for v in range(n):
        for h in range(int(D[v].max()) + 2):
            exact = sum(1 for w in range(n) if 0 <= D[v, w] <= h and client[w])
            assert g.hip_estimate(v, h, client) == float(exact)


def test_hip_unbiased_over_seeds():
    """E[N_hat(v, h)] = |ball| and E[predicated N_hat] = #clients in the ball:
    the HIP estimator is unbiased (Cohen 2014).  Mean over 1500 seeds must be
    within 4.5 standard errors for every (v, h) tested."""
    rowp, cols = small_er(60, 4.0, 6)
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    client = (np.arange(n) % 2 == 0).astype(np.uint8)
    k = 4
    probes = [(v, h) for v in (0, 7, 23, 41) for h in (1, 2, 3, 4, 6)]
    T = 1500
    vals = np.zeros((T, len(probes)))
    pvals = np.zeros((T, len(probes)))
    g = oracle.Graph(rowp, cols)
    for t in range(T):
        g.build_sketches(k, 1000 + t)
        for j, (v, h) in enumerate(probes):
            vals[t, j] = g.hip_estimate(v, h)
            pvals[t, j] = g.hip_estimate(v, h, client)
    for j, (v, h) in enumerate(probes):
        exact = sum(1 for w in range(n) if 0 <= D[v, w] <= h)
        exact_c = sum(1 for w in range(n) if 0 <= D[v, w] <= h and client[w])
        for arr, ex in ((vals[:, j], exact), (pvals[:, j], exact_c)):
            se = arr.std(ddof=1) / math.sqrt(T)
            assert abs(arr.mean() - ex) <= 4.5 * se + 1e-9, (v, h, arr.mean(), ex, se)


# ---------------------------------------------------------------- radius

def test_radius_complete_graph_closed_form():
    """K_n, all clients, n < k: r = c for c <= 1, else 1 + (c-1)/n."""
    for n in (3, 5, 9):
        rowp, cols = complete_graph(n)
        g = oracle.Graph(rowp, cols)
        g.build_sketches(16, 1)
        for c in (0.5, 1.0, 2.0, 7.5, 40.0):
            r = g.radii(np.full(n, c), np.ones(n, np.uint8))
            want = c if c <= 1 else 1 + (c - 1) / n
            assert np.allclose(r, want, rtol=1e-14, atol=0)


@pytest.mark.parametrize("name", ["path9", "star7", "cycle11", "mixed", "k6"])
def test_radius_exact_counts_equal_exact_root(name):
    """With exact counts (balls < k) the radius is the exact root of
    sum_c max(0, r - d(c,f)) = c(f) (Eq. 1, epsilon -> 0)."""
    rowp, cols = TINY[name]
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    client = (np.arange(n) % 4 != 3).astype(np.uint8)
    cost = np.array([1.5 + 3.25 * (v % 5) for v in range(n)])
    cost[2] = np.inf          # not a facility
    g = oracle.Graph(rowp, cols)
    g.build_sketches(16, 9)
    r = g.radii(cost, client)
    for f in range(n):
        if not np.isfinite(cost[f]):
            assert r[f] == np.inf
            continue
        ds = [D[f, c] for c in range(n) if client[c] and D[f, c] >= 0]
        want = brute.exact_radius(ds, cost[f])
        if want is None:
            assert r[f] == np.inf
        else:
            assert abs(r[f] - float(want)) <= 1e-12 * float(want), (f, r[f], want)


def test_radius_star_hand_computed():
    """Star with 4 leaves, all clients.  Centre: N_0=1, N_1=5 ->
    r = c (c<=1) else 1+(c-1)/5.  Leaf: N_0=1, N_1=2, N_2=5 ->
    r = c (c<=1); 1+(c-1)/2 (c<=3); 2+(c-3)/5."""
    rowp, cols = star_graph(4)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(16, 1)
    for c in (0.75, 2.0, 3.0, 10.0):
        r = g.radii(np.full(5, c), np.ones(5, np.uint8))
        centre = c if c <= 1 else 1 + (c - 1) / 5
        leaf = c if c <= 1 else (1 + (c - 1) / 2 if c <= 3 else 2 + (c - 3) / 5)
        assert r[0] == pytest.approx(centre, rel=1e-15)
        assert np.allclose(r[1:], leaf, rtol=1e-15)


def test_radius_residual_with_estimates():
    """For any ADS, r_f solves g(r_f) = c(f) for the estimated client counts:
    recompute g from the exported ADS groups and check the residual."""
    rowp, cols = flsynth.rmat(11, 8, 3)
    n = len(rowp) - 1
    client = flsynth.bernoulli(n, 4, 0.6)
    cost = flsynth.loguniform(n, 5, 5.0, 500.0)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(8, 1)
    A = g.ads()
    r = g.radii(cost, client)
    checked = 0
    for f in range(0, n, 5):
        if not np.isfinite(r[f]):
            continue
        W = {}
        for gi in range(A["gofs"][f], A["gofs"][f + 1]):
            e0 = A["eofs"][f] + (A["gcnt"][A["gofs"][f]:gi]).sum()
            ids = A["eid"][e0:e0 + A["gcounted"][gi]]
            W[int(A["ghop"][gi])] = client[ids].sum() * A["gwt"][gi]
        gval = sum(w * max(0.0, r[f] - h) for h, w in W.items())
        assert abs(gval - cost[f]) <= 1e-9 * cost[f]
        checked += 1
    assert checked > 50


# ---------------------------------------------------------------- MIS

@pytest.mark.parametrize("name", sorted(TINY))
def test_mis_is_lexicographically_first_on_materialised_hbar(name):
    """Open set = lexicographically-first MIS of the materialised conflict
    graph H-bar under key (r_f, pi_f) (Algorithm 3 and Section 4.3)."""
    rowp, cols = TINY[name]
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    client = (np.arange(n) % 3 != 2).astype(np.uint8)
    cost = np.array([2.0 + (7 * v % 11) for v in range(n)], float)
    cost[n // 2] = np.inf
    seed = 21
    g = oracle.Graph(rowp, cols)
    g.build_sketches(4, seed)
    r = g.radii(cost, client)
    op, nopen = g.open_facilities(r, client, seed)
    cand, balls, adj = brute.conflict_graph(D, r, client)
    key = lambda f: (r[f], oracle.priority(seed, f))
    S = brute.lfmis(cand, adj, key)
    assert set(np.flatnonzero(op)) == S and nopen == len(S)
    # independence, and every other candidate has a smaller-key neighbour in S
    for f in S:
        assert not (adj[f] & S)
    for f in cand:
        if f not in S:
            assert any(key(s) < key(f) for s in adj[f] & S)
    # each client is claimed by at most one open facility (Section 4.1)
    for c in range(n):
        if client[c]:
            assert sum(1 for f in S if c in balls[f]) <= 1


def test_mis_every_component_with_a_candidate_opens_one():
    rowp, cols = TINY["mixed"]
    n = len(rowp) - 1
    client = np.ones(n, np.uint8)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(4, 1)
    r = g.radii(np.full(n, 3.0), client)
    op, _ = g.open_facilities(r, client, 1)
    D = brute.apsp(rowp, cols)
    comps = {tuple(np.flatnonzero(D[v] >= 0)) for v in range(n)}
    for comp in comps:
        assert op[list(comp)].sum() >= 1


# ---------------------------------------------------------------- assignment

@pytest.mark.parametrize("name", sorted(TINY))
def test_assignment_is_nearest_open_facility_min_id(name):
    rowp, cols = TINY[name]
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    op = np.zeros(n, np.uint8)
    op[[v for v in range(n) if v % 4 == 1]] = 1
    g = oracle.Graph(rowp, cols)
    a, d = g.assign(op)
    wa, wd = brute.nearest_assignment(D, set(np.flatnonzero(op)))
    assert (d == wd).all() and (a == wa).all()


@pytest.mark.parametrize("name", sorted(TINY))
def test_nearest_open_single_source_matches_brute_force(name):
    """The per-vertex nearest-open-facility BFS (used to check sampled
    clients at full size) against all-pairs BFS: smallest distance, then
    smallest id; -1 where no open facility is reachable."""
    rowp, cols = TINY[name]
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    op = np.zeros(n, np.uint8)
    op[[v for v in range(n) if v % 3 == 2]] = 1
    g = oracle.Graph(rowp, cols)
    wa, wd = brute.nearest_assignment(D, set(np.flatnonzero(op)))
    for v in range(n):
        assert g.nearest_open(op, v) == (wa[v], wd[v])


@pytest.mark.parametrize("seed", [1, 2])
def test_radius_of_single_vertex_ads_equals_build_radius(seed):
    """The radius read off one vertex's Algorithm-1 ADS (used to check
    sampled facilities at full size) equals the radius of the hop-
    synchronous build, for every vertex: the two ADS constructions agree and
    feed the same shell walk."""
    w = flsynth.small_er(200, 3.0, 40 + seed, k=4, cost=5.0, client_p=0.6, fac_p=0.5)
    w.cost = np.where(np.isfinite(w.cost), flsynth.loguniform(w.n, seed, 2.0, 30.0), np.inf)
    g = oracle.Graph(w.rowp, w.cols)
    g.build_sketches(w.k, w.seed)
    r = g.radii(w.cost, w.client)
    for v in range(w.n):
        rv = oracle.radius_of_ads(g.vertex_ads(w.k, w.seed, v), w.client, w.cost[v])
        assert rv == r[v] or (math.isinf(rv) and math.isinf(r[v]))


def test_objective_recomputed_from_definition():
    rowp, cols = TINY["mixed"]
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    client = np.array([1, 1, 0, 1, 1, 1, 1, 1, 0, 1], np.uint8)
    cost = np.arange(1, n + 1, dtype=float) * 1.25
    op = np.zeros(n, np.uint8)
    op[[1, 5]] = 1
    g = oracle.Graph(rowp, cols)
    _, d = g.assign(op)
    obj, ds, un = oracle.objective(op, cost, client, d)
    served = [c for c in range(n) if client[c] and min(D[c, f] if D[c, f] >= 0 else 99 for f in (1, 5)) < 99]
    want_ds = sum(min(D[c, f] for f in (1, 5) if D[c, f] >= 0) for c in served)
    assert ds == want_ds
    assert un == sum(1 for c in range(n) if client[c]) - len(served)
    assert obj == cost[1] + cost[5] + want_ds


def test_full_solve_runs_on_er10k():
    """The whole oracle path finishes on the 10^4-vertex ER workload and its
    outputs satisfy the cross-step invariants."""
    w = flsynth.config("er10k")
    out = oracle.solve(w.rowp, w.cols, w.k, w.seed, w.cost, w.client)
    assert out["hops"] >= 3
    assert out["n_open"] > 0
    assert out["n_unserved"] == 0 or (out["dist"][w.client > 0] < 0).sum() == out["n_unserved"]
    assert (out["assign"][out["open"] > 0] == np.flatnonzero(out["open"])).all()


@pytest.mark.parametrize("name", sorted(TINY))
def test_mis_check_accepts_exactly_the_lexicographically_first_mis(name):
    """The parallel characterisation check (independent; every other
    candidate conflicts with an earlier member) accepts the brute-force
    lexicographically-first MIS of the materialised H-bar and rejects every
    set that differs from it by one facility."""
    rowp, cols = TINY[name]
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    client = (np.arange(n) % 3 != 1).astype(np.uint8)
    cost = np.array([1.5 + (5 * v % 7) for v in range(n)], float)
    seed = 33
    g = oracle.Graph(rowp, cols)
    g.build_sketches(4, seed)
    r = g.radii(cost, client)
    cand, _, adj = brute.conflict_graph(D, r, client)
    S = brute.lfmis(cand, adj, lambda f: (r[f], oracle.priority(seed, f)))
    op = np.zeros(n, np.uint8)
    op[list(S)] = 1
    assert g.check_open_facilities(r, client, seed, op) == (True, -1)
    for f in cand:
        flipped = op.copy()
        flipped[f] ^= 1
        ok, bad = g.check_open_facilities(r, client, seed, flipped)
        assert not ok and bad >= 0, f


@pytest.mark.parametrize("scale,const_cost", [(11, False), (12, True)])
def test_mis_check_agrees_with_the_greedy_on_rmat(scale, const_cost):
    """On R-MAT graphs (hubs; equal radii when every cost is the same, so the
    priorities decide) the greedy's set passes and one-facility changes fail."""
    rowp, cols = flsynth.rmat(scale, 8, 40 + scale)
    n = len(rowp) - 1
    client = flsynth.bernoulli(n, 41, 0.5)
    fac = flsynth.bernoulli(n, 42, 0.3)
    cost = np.where(fac > 0, 25.0 if const_cost else flsynth.loguniform(n, 43, 5.0, 500.0), np.inf)
    g = oracle.Graph(rowp, cols)
    g.build_sketches(16, 7)
    r = g.radii(cost, client)
    op, nopen = g.open_facilities(r, client, 7)
    assert nopen > 3
    assert g.check_open_facilities(r, client, 7, op) == (True, -1)
    members = np.flatnonzero(op)
    others = np.flatnonzero((op == 0) & np.isfinite(r))
    for f in list(members[:5]) + list(others[:5]):
        flipped = op.copy()
        flipped[f] ^= 1
        assert not g.check_open_facilities(r, client, 7, flipped)[0], f
    # another seed's priorities give another set (when it differs, it fails here)
    op2, _ = g.open_facilities(r, client, 8)
    if not np.array_equal(op2, op):
        assert not g.check_open_facilities(r, client, 7, op2)[0]
