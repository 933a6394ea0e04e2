"""GPU parity of the opening phase with eps > 0 (Section 4.1, Algorithm 3;
Section 4.2, Algorithms 4-5 and Eq. 2/3) and the selection of Algorithm 6
(Section 4.3), through the C ABI, against the oracle.

Bit-exact: the iteration at which every facility opened and every client
froze, gamma and alpha_0, the last iteration, the selected set, the
assignment and distances; objective within 1e-9 relative.  The GPU jumps
from event to event where the oracle runs every iteration of the grid, so
these cases also check that the jumps land where the iterations do."""
import numpy as np
import pytest

import brute
import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu

RTOL = 1e-9
EPS = (0.01, 0.1, 1.0)


def _inputs(n, seed, fac_p=0.5, cli_p=0.7, lo=0.5, hi=9.0):
    fac = flsynth.bernoulli(n, seed, fac_p)
    cost = np.where(fac > 0, flsynth.loguniform(n, seed + 1, lo, hi), np.inf)
    client = flsynth.bernoulli(n, seed + 2, cli_p)
    return cost, client


def _compare(rowp, cols, k, seed, eps, cost, client):
    want = oracle.solve_eps(rowp, cols, k, seed, eps, cost, client)
    got = fl.solve_eps(rowp, cols, k, seed, eps, cost, client)
    o, st = want["opening"], got["stats"]
    assert st["gamma"] == o["gamma"] and st["alpha0"] == o["alpha0"]
    assert st["iterations"] == o["iterations"]
    assert np.array_equal(got["fac_iter"], o["fac_iter"])
    assert np.array_equal(got["cli_iter"], o["cli_iter"])
    assert got["n_open"] == want["n_open"]
    assert np.array_equal(got["open"], want["open"])
    assert np.array_equal(got["dist"], want["dist"])
    assert np.array_equal(got["assign"], want["assign"])
    assert got["dist_sum"] == want["dist_sum"] and got["n_unserved"] == want["n_unserved"]
    assert abs(got["objective"] - want["objective"]) <= RTOL * abs(want["objective"])
    got["solve"].close()
    got["graph"].close()
    want["graph"].close()
    return got, want


@pytest.mark.parametrize("eps", EPS)
@pytest.mark.parametrize("kind", ["path", "star", "two", "er24"])
def test_tiny_graphs_exact_sketches(kind, eps):
    if kind == "path":
        rowp, cols = brute.csr_from_edges(14, [(i, i + 1) for i in range(13)])
    elif kind == "star":
        rowp, cols = brute.csr_from_edges(11, [(0, i) for i in range(1, 11)])
    elif kind == "two":
        rowp, cols = brute.csr_from_edges(14, [(i, i + 1) for i in range(7)] + [(8 + i, 9 + i) for i in range(5)])
    else:
        w = flsynth.small_er(24, 2.6, 41)
        rowp, cols = w.rowp, w.cols
    n = len(rowp) - 1
    cost, client = _inputs(n, 600)
    if kind == "two":
        cost[8:] = np.inf
    _compare(rowp, cols, 32, 7, eps, cost, client)


@pytest.mark.parametrize("eps", EPS)
@pytest.mark.parametrize("k", [4, 16])
def test_er_with_hip_estimates(k, eps):
    w = flsynth.small_er(2000, 6.0, 91)
    cost, client = _inputs(w.n, 900, fac_p=0.4, cli_p=0.5, lo=5.0, hi=200.0)
    got, _ = _compare(w.rowp, w.cols, k, 1, eps, cost, client)
    assert got["n_open"] > 3 and got["stats"]["events"] >= 2


@pytest.mark.parametrize("eps", EPS)
def test_rmat_with_hubs(eps):
    rowp, cols = flsynth.rmat(14, 16, 77)
    n = len(rowp) - 1
    cost, client = _inputs(n, 950, fac_p=0.3, cli_p=0.6, lo=5.0, hi=500.0)
    got, _ = _compare(rowp, cols, 16, 3, eps, cost, client)
    assert got["stats"]["groups"] >= 1


def test_device_memory_and_edge_cases():
    torch = pytest.importorskip("torch")
    w = flsynth.small_er(500, 5.0, 95)
    cost, client = _inputs(w.n, 960, fac_p=0.5, cli_p=0.5, lo=2.0, hi=50.0)
    g = fl.Graph(w.rowp, w.cols)
    g.build_sketches(16, 2)
    s = fl.Solve(g)
    dev = torch.device("cuda:0")
    op = torch.zeros(w.n, dtype=torch.uint8, device=dev)
    fi = torch.zeros(w.n, dtype=torch.int32, device=dev)
    ci = torch.zeros(w.n, dtype=torch.int32, device=dev)
    _, n_open, _, _ = s.open_facilities_eps(0.1, torch.from_numpy(cost).to(dev), torch.from_numpy(client).to(dev),
                                            op, fi, ci)
    want = oracle.solve_eps(w.rowp, w.cols, 16, 2, 0.1, cost, client)
    assert n_open == want["n_open"]
    assert np.array_equal(op.cpu().numpy(), want["open"])
    assert np.array_equal(fi.cpu().numpy(), want["opening"]["fac_iter"])
    assert np.array_equal(ci.cpu().numpy(), want["opening"]["cli_iter"])
    # assignment and objective follow the selected set
    a, d = s.assign_clients()
    assert np.array_equal(a, want["assign"]) and np.array_equal(d, want["dist"])
    # no clients: nothing opens, nobody is assigned
    op2, n2, fi2, ci2 = s.open_facilities_eps(0.1, cost, np.zeros(w.n, np.uint8))
    assert n2 == 0 and (fi2 == -1).all() and (ci2 == -1).all()
    # bad eps and bad costs
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(fl.FLError) as e:
            s.open_facilities_eps(bad, cost, client)
        assert e.value.status == fl.FL_EINVAL
    bad_cost = cost.copy()
    bad_cost[np.flatnonzero(np.isfinite(cost))[0]] = -3.0
    with pytest.raises(fl.FLError):
        s.open_facilities_eps(0.1, bad_cost, client)
    s.close()
    g.close()
