"""Pins of the oracle's opening phase with epsilon > 0 (Section 4.1,
Algorithm 3; Section 4.2, Algorithms 4-5 and Eq. 2/3; Section 4.3,
Algorithm 6).

* gamma against its definition on all-pairs distances;
* the whole opening loop (which facility opens and which client freezes at
  which iteration, and q(f)) against an independent restatement on exact
  distances (tests/brute.py), with k above the vertex count so that the
  ADS holds every vertex with weight 1;
* the closed form of q(f) against the literal incremental Eq. 2/3, with
  HIP estimates (small k), for eps in {0.01, 0.1, 1};
* the selection against the lexicographically-first MIS under pi of the
  materialised H-bar, and its independence and maximality;
* edge cases: no clients, no facilities, a component without facilities,
  a facility that is its own client.
Planted mistakes (a dropped (1 + eps), freezing at radius alpha instead of
(1 + eps) alpha, a shell rounded down) fail the brute-force comparison."""
import numpy as np
import pytest

import brute
import flsynth
import oracle

RTOL = 1e-9


def _graph(kind, seed):
    if kind == "path":
        return brute.csr_from_edges(14, [(i, i + 1) for i in range(13)])
    if kind == "star":
        return brute.csr_from_edges(11, [(0, i) for i in range(1, 11)])
    if kind == "two":  # two components, the second without facilities below
        e = [(i, i + 1) for i in range(7)] + [(8 + i, 9 + i) for i in range(5)]
        return brute.csr_from_edges(14, e)
    w = flsynth.small_er(24, 2.6, seed)
    return w.rowp, w.cols


def _inputs(n, seed, fac_p=0.5, cli_p=0.7, lo=0.5, hi=9.0):
    fac = flsynth.bernoulli(n, seed, fac_p)
    cost = np.where(fac > 0, flsynth.loguniform(n, seed + 1, lo, hi), np.inf)
    client = flsynth.bernoulli(n, seed + 2, cli_p)
    return cost, client


@pytest.mark.parametrize("kind,seed", [("er", 31), ("er", 32), ("path", 0), ("star", 0), ("two", 0)])
def test_gamma_matches_its_definition(kind, seed):
    rowp, cols = _graph(kind, seed)
    n = len(rowp) - 1
    cost, client = _inputs(n, 500 + seed)
    og = oracle.Graph(rowp, cols)
    assert og.eps_gamma(cost, client) == brute.eps_gamma(brute.apsp(rowp, cols), cost, client)


@pytest.mark.parametrize("eps", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("kind,seed", [("er", 41), ("er", 42), ("er", 43), ("path", 0), ("star", 0), ("two", 0)])
def test_opening_loop_matches_exact_distances(kind, seed, eps):
    rowp, cols = _graph(kind, seed)
    n = len(rowp) - 1
    cost, client = _inputs(n, 600 + seed)
    if kind == "two":
        cost[8:] = np.inf  # the second component has clients but no facility
    D = brute.apsp(rowp, cols)
    want = brute.eps_opening(D, cost, client, eps)
    og = oracle.Graph(rowp, cols)
    og.build_sketches(32, 7)  # k > n: every vertex in the ADS, weight 1
    got = og.eps_open(eps, cost, client)
    assert got["alpha0"] == want["alpha0"]
    assert got["iterations"] == want["iterations"]
    assert np.array_equal(got["fac_iter"], want["fac_iter"])
    assert np.array_equal(got["cli_iter"], want["cli_iter"])
    fac = np.isfinite(cost)
    assert np.allclose(got["q"][fac], want["q"][fac], rtol=RTOL, atol=1e-12)
    if kind == "two":
        assert (got["cli_iter"][8:] == -1).all()
    # every opened facility reached its cost, and no client froze before a
    # facility within (1 + eps) alpha opened
    assert (got["q"][got["fac_iter"] >= 0] >= cost[got["fac_iter"] >= 0]).all()


@pytest.mark.parametrize("eps", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("k", [4, 16])
def test_closed_form_matches_literal_eq2_eq3(eps, k):
    w = flsynth.small_er(300, 4.0, 77)
    cost, client = _inputs(w.n, 700, fac_p=0.3, cli_p=0.6, lo=2.0, hi=60.0)
    og = oracle.Graph(w.rowp, w.cols)
    og.build_sketches(k, 3)
    a = og.eps_open(eps, cost, client, mode=0)
    b = og.eps_open(eps, cost, client, mode=1)
    assert np.array_equal(a["fac_iter"], b["fac_iter"])
    assert np.array_equal(a["cli_iter"], b["cli_iter"])
    fac = np.isfinite(cost)
    assert np.allclose(a["q"][fac], b["q"][fac], rtol=RTOL, atol=1e-9)
    assert (a["fac_iter"] >= 0).sum() > 3 and (a["cli_iter"] >= 0).sum() > 10


@pytest.mark.parametrize("eps", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("seed", [51, 52, 53])
def test_selection_is_lexicographically_first_mis_of_hbar(eps, seed):
    rowp, cols = _graph("er", seed)
    n = len(rowp) - 1
    cost, client = _inputs(n, 800 + seed, fac_p=0.7, cli_p=0.9, lo=0.3, hi=4.0)
    og = oracle.Graph(rowp, cols)
    og.build_sketches(32, 5)
    o = og.eps_open(eps, cost, client)
    op, nopen = og.eps_select(eps, o["alpha0"], o["fac_iter"], o["cli_iter"], 5)
    D = brute.apsp(rowp, cols)
    opened, adj = brute.eps_hbar(D, eps, o["alpha0"], o["fac_iter"], o["cli_iter"])
    pi = {f: oracle.priority(5, f) for f in opened}
    S = brute.lfmis(opened, adj, key=lambda f: pi[f])
    assert set(np.flatnonzero(op)) == S and nopen == len(S)
    for f in opened:  # independent and maximal
        if f in S:
            assert not (adj[f] & S)
        else:
            assert any(pi[g] < pi[f] for g in adj[f] & S)


def test_edge_cases():
    rowp, cols = _graph("path", 0)
    n = len(rowp) - 1
    og = oracle.Graph(rowp, cols)
    og.build_sketches(16, 1)
    none = og.eps_open(0.1, np.full(n, 5.0), np.zeros(n, np.uint8))
    assert (none["fac_iter"] == -1).all() and none["iterations"] == 0
    none = og.eps_open(0.1, np.full(n, np.inf), np.ones(n, np.uint8))
    assert (none["fac_iter"] == -1).all() and none["iterations"] == 0
    # a single facility that is also the only client: q = (1 + eps) alpha - alpha_0
    cost = np.full(n, np.inf)
    cost[3] = 2.0
    client = np.zeros(n, np.uint8)
    client[3] = 1
    o = og.eps_open(0.5, cost, client)
    assert o["fac_iter"][3] >= 1 and o["cli_iter"][3] == o["fac_iter"][3]
    assert o["gamma"] == 2.0
    op, no = og.eps_select(0.5, o["alpha0"], o["fac_iter"], o["cli_iter"], 1)
    assert no == 1 and op[3] == 1


def test_whole_path_serves_every_reachable_client():
    w = flsynth.small_er(2000, 6.0, 91)
    cost, client = _inputs(w.n, 900, fac_p=0.4, cli_p=0.5, lo=5.0, hi=200.0)
    for eps in (0.01, 0.1, 1.0):
        r = oracle.solve_eps(w.rowp, w.cols, 16, 1, eps, cost, client)
        o = r["opening"]
        assert r["n_open"] > 0
        # the selection keeps a subset of the opened facilities
        assert (r["open"] <= (o["fac_iter"] >= 0)).all()
        D_any = r["dist"]
        reach = brute_reach(w, cost, client)
        assert ((D_any >= 0) | ~reach).all()


def brute_reach(w, cost, client):
    """Clients whose component holds a facility (by BFS labels)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    A = sp.csr_matrix((np.ones(len(w.cols)), w.cols, w.rowp), shape=(w.n, w.n))
    _, lab = connected_components(A, directed=False)
    has = np.zeros(lab.max() + 1, bool)
    has[lab[np.isfinite(cost)]] = True
    return (client > 0) & has[lab]
