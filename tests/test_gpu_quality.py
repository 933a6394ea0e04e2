"""Quality of the GPU path against the oracle's references (Section 5.2
compares the method's cost with a sequential local search, Table 2): on
instances small enough to enumerate, the GPU's open set serves every client
a facility can reach, its objective is the cost of that set by definition,
and it is at least the optimum; bench.py --workload quality reports the
ratios."""
import numpy as np
import pytest

import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu


def _instance(seed, n=16):
    w = flsynth.small_er(n, 2.2, 40 + seed)
    cost = flsynth.loguniform(n, 50 + seed, 0.5, 12.0)
    client = flsynth.bernoulli(n, 60 + seed, 0.85)
    return w.rowp, w.cols, cost, client


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("exact", [False, True])
def test_gpu_solution_against_the_optimum(seed, exact):
    rowp, cols, cost, client = _instance(seed)
    g = fl.Graph(rowp, cols)
    g.build_sketches(32, 1)
    s = fl.Solve(g)
    if exact:
        s.compute_radii_exact(cost, client)
    else:
        s.compute_radii(cost, client)
    op, _ = s.open_facilities()
    s.assign_clients()
    obj, _, _ = s.objective()
    s.close()
    g.close()
    orc = oracle.Graph(rowp, cols)
    c = orc.fl_cost(cost, client, op)
    assert np.isfinite(c)
    assert abs(c - obj) <= 1e-12 * obj
    _, opt = orc.optimum(cost, client)
    assert c >= opt * (1 - 1e-12)
    # local search started from the GPU's set never ends above it
    _, ls, _ = orc.local_search(cost, client, start=op)
    assert ls <= c * (1 + 1e-12)
