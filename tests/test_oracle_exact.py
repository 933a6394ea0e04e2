"""Pins for the oracle's exact neighbourhood sizes and exact radii (the
ground truth of the ADS accuracy study, Section 5.1 "Accuracy vs. k",
Fig. 1): checked against scipy's breadth-first shortest paths, closed forms,
the exact root of Eq. 1 at epsilon -> 0 (rational arithmetic), and the
sketch radius where the sketches are exact.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import brute
import flsynth
import oracle


def _scipy_dist(rowp, cols):
    n = len(rowp) - 1
    A = sp.csr_matrix((np.ones(len(cols)), cols, rowp), shape=(n, n))
    D = shortest_path(A, method="D", unweighted=True, directed=False)
    D[np.isinf(D)] = -1
    return D.astype(np.int64)


def _graphs():
    out = {}
    w = flsynth.small_er(300, 3.0, 41)  # several components at this density
    out["er300"] = (w.rowp, w.cols)
    out["rmat9"] = flsynth.rmat(9, 8, 5)
    out["path40"] = brute.csr_from_edges(40, [(i, i + 1) for i in range(39)])
    out["star60"] = brute.csr_from_edges(61, [(0, i) for i in range(1, 61)])
    return out


GRAPHS = _graphs()


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("with_pred", [False, True])
def test_ball_sizes_match_scipy_bfs(name, with_pred):
    rowp, cols = GRAPHS[name]
    n = len(rowp) - 1
    D = _scipy_dist(rowp, cols)
    pred = flsynth.bernoulli(n, 77, 0.4) if with_pred else None
    rng = np.random.default_rng(3)
    src = rng.choice(n, size=min(n, 25), replace=False).astype(np.int32)
    H = 14
    g = oracle.Graph(rowp, cols)
    got = g.ball_sizes(src, H, pred)
    for i, v in enumerate(src):
        ok = D[v] >= 0
        if pred is not None:
            ok &= pred > 0
        for h in range(H + 1):
            assert got[i, h] == int(np.sum(ok & (D[v] <= h))), (name, v, h)


def test_ball_sizes_path_closed_form():
    """Path P_n: |Ball_h(v)| = min(v, h) + min(n-1-v, h) + 1."""
    n = 40
    rowp, cols = GRAPHS["path40"]
    g = oracle.Graph(rowp, cols)
    src = np.arange(n, dtype=np.int32)
    got = g.ball_sizes(src, 50)
    for v in range(n):
        for h in range(51):
            assert got[v, h] == min(v, h) + min(n - 1 - v, h) + 1


def test_ball_sizes_rejects_bad_sources():
    rowp, cols = GRAPHS["path40"]
    g = oracle.Graph(rowp, cols)
    with pytest.raises(RuntimeError):
        g.ball_sizes(np.array([40], np.int32), 3)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_exact_radius_is_the_exact_root(name):
    """r_f solves sum_{c in C} max(0, r - d(c, f)) = c(f) exactly (rational
    root from all-pairs distances), on graphs far larger than any sketch."""
    rowp, cols = GRAPHS[name]
    n = len(rowp) - 1
    D = _scipy_dist(rowp, cols)
    client = flsynth.bernoulli(n, 12, 0.6)
    cost = flsynth.loguniform(n, 13, 0.5, 300.0)
    cost[flsynth.bernoulli(n, 14, 0.2) > 0] = np.inf
    g = oracle.Graph(rowp, cols)
    r = g.exact_radii(cost, client)
    for f in range(n):
        if not np.isfinite(cost[f]):
            assert r[f] == np.inf
            continue
        ds = [D[f, c] for c in range(n) if client[c] and D[f, c] >= 0]
        want = brute.exact_radius(ds, cost[f])
        if want is None:
            assert r[f] == np.inf, f
        else:
            assert abs(r[f] - float(want)) <= 1e-12 * float(want), (name, f, r[f], float(want))


def test_exact_radius_closed_forms():
    """K_40 and a 60-leaf star, all clients, far beyond k: the walk's
    closed forms, evaluated in the same IEEE order (so compared with ==)."""
    n = 40
    rowp, cols = brute.csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    g = oracle.Graph(rowp, cols)
    for c in (0.25, 1.0, 3.5, 77.0):
        r = g.exact_radii(np.full(n, c), np.ones(n, np.uint8))
        want = c if c <= 1 else 1.0 + (c - 1.0) / n
        assert np.all(r == want)
    rowp, cols = GRAPHS["star60"]
    g = oracle.Graph(rowp, cols)
    m = 60
    for c in (0.5, 2.0, 3.0, 50.0):
        r = g.exact_radii(np.full(m + 1, c), np.ones(m + 1, np.uint8))
        centre = c if c <= 1 else 1.0 + (c - 1.0) / (m + 1)
        leaf = c if c <= 1 else (1.0 + (c - 1.0) / 2 if c <= 3 else 2.0 + (c - 3.0) / (m + 1))
        assert r[0] == centre
        assert np.all(r[1:] == leaf)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_radius_equals_sketch_radius_when_sketches_are_exact(seed):
    """With k >= n every HIP weight is 1 and the sketch radius walks the same
    numbers: the two radii are identical bit for bit."""
    w = flsynth.small_er(30, 2.5, 100 + seed)
    n = 30
    client = flsynth.bernoulli(n, 200 + seed, 0.7)
    cost = flsynth.loguniform(n, 300 + seed, 0.3, 60.0)
    g = oracle.Graph(w.rowp, w.cols)
    g.build_sketches(32, seed)
    assert np.array_equal(g.radii(cost, client), g.exact_radii(cost, client))
    # and the HIP estimates are the exact sizes
    src = np.arange(n, dtype=np.int32)
    exact = g.ball_sizes(src, 8, client)
    for v in range(n):
        for h in range(9):
            assert g.hip_estimate(v, h, client) == float(exact[v, h])


def test_exact_radii_of_a_sample_match_all():
    rowp, cols = GRAPHS["rmat9"]
    n = len(rowp) - 1
    client = flsynth.bernoulli(n, 5, 0.5)
    cost = flsynth.loguniform(n, 6, 1.0, 100.0)
    g = oracle.Graph(rowp, cols)
    every = g.exact_radii(cost, client)
    sample = np.array([0, 7, n - 1, 100, 3], np.int32)
    assert np.array_equal(g.exact_radii(cost, client, sample), every[sample])
