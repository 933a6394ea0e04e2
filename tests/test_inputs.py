"""The seeded input recipes (flsynth) on the CPU: the graphs are simple,
symmetric CSR with the stated sizes, the draws are reproducible and follow
their distributions, and the named workloads match their recipes."""
import math

import numpy as np
import pytest

import flsynth


def _check_simple_symmetric(rowp, cols, n):
    assert rowp.dtype == np.int64 and cols.dtype == np.int32
    assert len(rowp) == n + 1 and rowp[0] == 0 and rowp[-1] == len(cols)
    assert np.all(np.diff(rowp) >= 0)
    assert np.all((cols >= 0) & (cols < n))
    src = np.repeat(np.arange(n), np.diff(rowp))
    assert not np.any(src == cols)  # no self-loops
    key = src.astype(np.int64) * n + cols
    assert len(np.unique(key)) == len(key)  # no duplicate entries
    rev = cols.astype(np.int64) * n + src
    assert np.array_equal(np.sort(key), np.sort(rev))  # (u, v) present iff (v, u) is
    return src


def test_er_is_g_n_m():
    rowp, cols = flsynth.er(500, 1500, 7)
    _check_simple_symmetric(rowp, cols, 500)
    assert len(cols) == 3000  # M distinct undirected pairs
    r2, c2 = flsynth.er(500, 1500, 7)
    assert np.array_equal(rowp, r2) and np.array_equal(cols, c2)
    r3, c3 = flsynth.er(500, 1500, 8)
    assert not np.array_equal(cols, c3)


@pytest.mark.parametrize("scale", [8, 12])
def test_rmat_is_simple_symmetric_and_skewed(scale):
    rowp, cols = flsynth.rmat(scale, 16, 3)
    n = 1 << scale
    _check_simple_symmetric(rowp, cols, n)
    nnz = len(cols)
    assert nnz <= 2 * 16 * n  # draws, symmetrised, deduplicated
    deg = np.diff(rowp)
    assert deg.max() > 8 * deg.mean()  # the (0.57, 0.19, 0.19, 0.05) recursion concentrates edges
    assert (deg == 0).any() or scale > 10  # small R-MAT graphs have isolated vertices
    r2, c2 = flsynth.rmat(scale, 16, 3)
    assert np.array_equal(rowp, r2) and np.array_equal(cols, c2)


def test_bernoulli_and_loguniform_follow_their_distributions():
    n = 200_000
    m = flsynth.bernoulli(n, 5, 0.3)
    assert set(np.unique(m)) <= {0, 1}
    assert abs(m.mean() - 0.3) < 0.01
    assert np.array_equal(m, flsynth.bernoulli(n, 5, 0.3))
    c = flsynth.loguniform(n, 6, 10.0, 1.0e4)
    assert c.min() >= 10.0 and c.max() <= 1.0e4
    lg = np.log(c)
    lo, hi = math.log(10.0), math.log(1.0e4)
    assert abs(lg.mean() - (lo + hi) / 2) < 0.02 * (hi - lo)  # uniform in log space
    assert abs(np.mean(lg < (lo + hi) / 2) - 0.5) < 0.01
    fac = flsynth.bernoulli(n, 7, 0.1)
    cf = flsynth.loguniform(n, 6, 10.0, 1.0e4, fac)
    assert np.all(np.isinf(cf[fac == 0])) and np.all(np.isfinite(cf[fac == 1]))


def test_edge_weights_symmetric_uniform_and_reproducible():
    rowp, cols = flsynth.rmat(12, 16, 9)
    n = len(rowp) - 1
    w = flsynth.edge_weights(rowp, cols, 5)
    src = np.repeat(np.arange(n), np.diff(rowp))
    assert w.dtype == np.int32 and w.min() >= 1 and w.max() <= 100
    key = src.astype(np.int64) * n + cols
    order = np.argsort(key)
    rkey = cols.astype(np.int64) * n + src
    rorder = np.argsort(rkey)
    assert np.array_equal(w[order], w[rorder])  # the same length in both directions
    und = w[src < cols]
    counts = np.bincount(und, minlength=101)[1:]
    exp = len(und) / 100
    assert np.all(np.abs(counts - exp) < 6 * math.sqrt(exp))  # every length about equally often
    assert np.array_equal(w, flsynth.edge_weights(rowp, cols, 5))
    assert not np.array_equal(w, flsynth.edge_weights(rowp, cols, 6))
    w3 = flsynth.edge_weights(rowp, cols, 5, 1, 3)
    assert set(np.unique(w3)) == {1, 2, 3}


def test_named_workload_er10k_matches_its_recipe():
    w = flsynth.config("er10k")
    assert w.n == 10_000 and w.nnz == 80_000 and w.k == 16
    assert np.all(w.cost == 20.0) and np.all(w.client == 1)
    _check_simple_symmetric(w.rowp, w.cols, w.n)


def test_scaled_rmat26_recipe():
    """The rmat26 recipe at a small scale: clients Bernoulli(0.5), facilities
    Bernoulli(0.1) with log-uniform costs in [10, 10^4], k = 16."""
    w = flsynth.config("rmat26s14")
    assert w.n == 1 << 14 and w.k == 16
    fac = np.isfinite(w.cost)
    assert abs(w.client.mean() - 0.5) < 0.03 and abs(fac.mean() - 0.1) < 0.02
    assert w.cost[fac].min() >= 10.0 and w.cost[fac].max() <= 1.0e4
    _check_simple_symmetric(w.rowp, w.cols, w.n)
