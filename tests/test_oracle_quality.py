"""Pins for the oracle's quality references (Section 5.2, Table 2 compares
the method's cost with a sequential local search): the cost of an open set,
the optimum by enumeration and the add/drop/swap local search, checked
against a separate Python enumeration over all-pairs distances, the
local-optimality conditions and the 3 x optimum bound of Arya et al. (2004).
"""
import itertools

import numpy as np
import pytest

import brute
import flsynth
import oracle


def _py_cost(D, cost, client, S):
    """Definition: sum_{f in S} c(f) + sum_c min_{f in S} d(c, f) over the
    clients some facility reaches; +inf if such a client is unserved."""
    fac = [f for f in range(len(cost)) if np.isfinite(cost[f])]
    total = 0.0
    for f in sorted(S):
        total = total + cost[f]
    ds = 0
    for c in range(len(cost)):
        if not client[c] or not any(D[f, c] >= 0 for f in fac):
            continue
        ds_c = [D[f, c] for f in S if D[f, c] >= 0]
        if not ds_c:
            return np.inf
        ds += min(ds_c)
    return total + float(ds)


def _instance(seed, n=11, p_fac=0.6):
    w = flsynth.small_er(n, 1.6, 900 + seed)  # sparse: several components
    cost = flsynth.loguniform(n, 910 + seed, 0.3, 9.0)
    cost[flsynth.bernoulli(n, 920 + seed, 1.0 - p_fac) > 0] = np.inf
    client = flsynth.bernoulli(n, 930 + seed, 0.8)
    return w.rowp, w.cols, cost, client


@pytest.mark.parametrize("seed", range(6))
def test_cost_and_optimum_match_enumeration(seed):
    rowp, cols, cost, client = _instance(seed)
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    g = oracle.Graph(rowp, cols)
    fac = [f for f in range(n) if np.isfinite(cost[f])]
    best = np.inf
    for r in range(1, len(fac) + 1):
        for S in itertools.combinations(fac, r):
            c = _py_cost(D, cost, client, S)
            best = min(best, c)
            mask = np.zeros(n, np.uint8)
            mask[list(S)] = 1
            if r <= 2 or r == len(fac):
                got = g.fl_cost(cost, client, mask)
                assert (got == c) or abs(got - c) <= 1e-12 * abs(c), (S, got, c)
    op, obj = g.optimum(cost, client)
    assert abs(obj - best) <= 1e-12 * best
    assert abs(_py_cost(D, cost, client, np.flatnonzero(op)) - best) <= 1e-12 * best


@pytest.mark.parametrize("seed", range(6))
def test_local_search_is_a_local_optimum_within_three_times_the_optimum(seed):
    rowp, cols, cost, client = _instance(seed, n=14, p_fac=0.8)
    n = len(rowp) - 1
    D = brute.apsp(rowp, cols)
    g = oracle.Graph(rowp, cols)
    _, opt = g.optimum(cost, client)
    op, obj, moves = g.local_search(cost, client)
    S = set(np.flatnonzero(op).tolist())
    assert abs(_py_cost(D, cost, client, S) - obj) <= 1e-12 * obj
    assert obj >= opt * (1 - 1e-12)
    assert obj <= 3.0 * opt * (1 + 1e-12)  # Arya et al.: add/drop/swap local optima
    fac = [f for f in range(n) if np.isfinite(cost[f])]
    closed = [f for f in fac if f not in S]
    tol = 1e-9 * obj
    for j in closed:
        assert _py_cost(D, cost, client, S | {j}) >= obj - tol, ("add", j)
    for i in S:
        assert _py_cost(D, cost, client, S - {i}) >= obj - tol, ("drop", i)
        for j in closed:
            assert _py_cost(D, cost, client, (S - {i}) | {j}) >= obj - tol, ("swap", i, j)


def test_local_search_from_a_given_start_and_move_cap():
    rowp, cols = flsynth.rmat(8, 8, 3)
    n = len(rowp) - 1
    cost = flsynth.loguniform(n, 4, 2.0, 40.0)
    client = np.ones(n, np.uint8)
    g = oracle.Graph(rowp, cols)
    every = np.isfinite(cost).astype(np.uint8)
    op, obj, moves = g.local_search(cost, client, start=every)
    assert moves > 0 and obj < g.fl_cost(cost, client, every)
    _, obj0, moves0 = g.local_search(cost, client, start=every, max_moves=0)
    assert moves0 == 0 and obj0 == g.fl_cost(cost, client, every)
