"""GPU parity of the exact-size and exact-radius calls (the ground truth of
the ADS accuracy study, Section 5.1, Fig. 1) against the CPU oracle:
exact ball sizes bit-exact, HIP estimates and exact-count radii bit-exact
(the kernels evaluate the oracle's FP64 operations in the oracle's order on
the same exact integers), and the exact-radius pipeline's open set,
assignment and objective as for the sketch pipeline.
"""
import numpy as np
import pytest

import brute
import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu


def _graphs():
    out = {}
    w = flsynth.small_er(3000, 3.0, 61)          # many components, short rows
    out["er3000"] = (w.rowp, w.cols)
    out["rmat12"] = flsynth.rmat(12, 16, 62)       # hubs: rows far longer than 32
    out["path300"] = brute.csr_from_edges(300, [(i, i + 1) for i in range(299)])
    out["star400"] = brute.csr_from_edges(401, [(0, i) for i in range(1, 401)])
    out["edgeless"] = (np.zeros(9, np.int64), np.zeros(0, np.int32))
    return out


GRAPHS = _graphs()


def _sources(n, m, seed):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=m).astype(np.int32)  # repeats allowed
    src[:3] = [0, n - 1, 0]
    return src


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("with_pred", [False, True])
def test_ball_sizes_match_oracle(name, with_pred):
    rowp, cols = GRAPHS[name]
    n = len(rowp) - 1
    src = _sources(n, 600, 7)  # three sweeps, the last one ragged
    pred = flsynth.bernoulli(n, 8, 0.35) if with_pred else None
    D = 12
    g = fl.Graph(rowp, cols)
    got = g.ball_sizes(src, D, pred)
    want = oracle.Graph(rowp, cols).ball_sizes(src, D, pred)
    assert got.dtype == np.int64 and got.shape == (len(src), D + 1)
    assert np.array_equal(got, want)
    g.close()


def test_ball_sizes_edge_cases_and_device_memory():
    import torch
    rowp, cols = GRAPHS["rmat12"]
    n = len(rowp) - 1
    g = fl.Graph(rowp, cols)
    orc = oracle.Graph(rowp, cols)
    # no sources
    assert g.ball_sizes(np.zeros(0, np.int32), 4).shape == (0, 5)
    # distance 0 only: the source itself (under the predicate)
    src = _sources(n, 300, 9)
    pred = flsynth.bernoulli(n, 10, 0.5)
    assert np.array_equal(g.ball_sizes(src, 0, pred)[:, 0], pred[src].astype(np.int64))
    # device arrays in and out
    src_d = torch.from_numpy(src).cuda()
    pred_d = torch.from_numpy(pred).cuda()
    out_d = torch.zeros((len(src), 7), dtype=torch.int64, device="cuda")
    g.ball_sizes(src_d, 6, pred_d, out=out_d)
    assert np.array_equal(out_d.cpu().numpy(), orc.ball_sizes(src, 6, pred))
    # ids outside [0, n) are refused
    with pytest.raises(fl.FLError):
        g.ball_sizes(np.array([0, n], np.int32), 3)
    with pytest.raises(fl.FLError):
        g.ball_sizes(np.array([-1], np.int32), 3)
    # estimates need the sketches
    with pytest.raises(fl.FLError):
        g.ball_estimates(src, 3)
    g.close()


@pytest.mark.parametrize("name", ["er3000", "rmat12", "star400"])
@pytest.mark.parametrize("k", [16, 32])
def test_ball_estimates_match_oracle_hip(name, k):
    rowp, cols = GRAPHS[name]
    n = len(rowp) - 1
    seed = 4
    src = _sources(n, 200, 11)
    pred = flsynth.bernoulli(n, 12, 0.6)
    D = 9
    g = fl.Graph(rowp, cols)
    g.build_sketches(k, seed)
    orc = oracle.Graph(rowp, cols)
    orc.build_sketches(k, seed)
    for p in (None, pred):
        got = g.ball_estimates(src, D, p)
        for i, v in enumerate(src):
            for h in range(D + 1):
                assert got[i, h] == orc.hip_estimate(int(v), h, p), (name, k, v, h)
    g.close()


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_exact_radii_match_oracle(name):
    rowp, cols = GRAPHS[name]
    n = len(rowp) - 1
    client = flsynth.bernoulli(n, 21, 0.55)
    cost = flsynth.loguniform(n, 22, 0.3, 400.0)
    cost[flsynth.bernoulli(n, 23, 0.3) > 0] = np.inf
    g = fl.Graph(rowp, cols)
    g.build_sketches(16, 3)
    s = fl.Solve(g)
    r = s.compute_radii_exact(cost, client)
    want = oracle.Graph(rowp, cols).exact_radii(cost, client)
    assert np.array_equal(r.view(np.uint64), want.view(np.uint64))
    s.close()
    g.close()


@pytest.mark.parametrize("name", ["er3000", "rmat12"])
def test_exact_radius_pipeline_matches_oracle(name):
    """Exact radii, then the MIS, assignment and objective on them."""
    rowp, cols = GRAPHS[name]
    n = len(rowp) - 1
    seed = 5
    client = flsynth.bernoulli(n, 31, 0.5)
    cost = flsynth.loguniform(n, 32, 1.0, 200.0)
    g = fl.Graph(rowp, cols)
    g.build_sketches(16, seed)
    s = fl.Solve(g)
    r = s.compute_radii_exact(cost, client)
    op, nopen = s.open_facilities()
    a, d = s.assign_clients()
    obj, ds, un = s.objective()
    orc = oracle.Graph(rowp, cols)
    r_o = orc.exact_radii(cost, client)
    op_o, nopen_o = orc.open_facilities(r_o, client, seed)
    a_o, d_o = orc.assign(op_o)
    obj_o, ds_o, un_o = oracle.objective(op_o, cost, client, d_o)
    assert np.array_equal(r, r_o)
    assert nopen == nopen_o and np.array_equal(op, op_o)
    assert np.array_equal(a, a_o) and np.array_equal(d, d_o)
    assert (ds, un) == (ds_o, un_o)
    assert abs(obj - obj_o) <= 1e-9 * abs(obj_o)
    # the sketch radii of the same solve are still available afterwards
    r_sk = s.compute_radii(cost, client)
    assert np.array_equal(r_sk, orc_sketch_radii(rowp, cols, 16, seed, cost, client))
    s.close()
    g.close()


def orc_sketch_radii(rowp, cols, k, seed, cost, client):
    o = oracle.Graph(rowp, cols)
    o.build_sketches(k, seed)
    return o.radii(cost, client)


@pytest.mark.parametrize("seed", [1, 2])
def test_exact_and_sketch_radii_agree_when_k_covers_the_graph(seed):
    w = flsynth.small_er(30, 2.5, 500 + seed)
    n = 30
    client = flsynth.bernoulli(n, 600 + seed, 0.7)
    cost = flsynth.loguniform(n, 700 + seed, 0.3, 60.0)
    g = fl.Graph(w.rowp, w.cols)
    g.build_sketches(32, seed)
    s = fl.Solve(g)
    assert np.array_equal(s.compute_radii(cost, client), s.compute_radii_exact(cost, client))
    src = np.arange(n, dtype=np.int32)
    assert np.array_equal(g.ball_estimates(src, 8, client), g.ball_sizes(src, 8, client).astype(np.float64))
    s.close()
    g.close()


def test_exact_on_the_s20_graph_sampled():
    """R-MAT scale 20 (the 1M-vertex recipe): exact sizes of 300 sampled
    vertices to distance 6, and exact radii of 2,000 sampled facilities,
    against the oracle's BFS."""
    w = flsynth.config("rmat20")
    n = w.n
    rng = np.random.default_rng(77)
    src = rng.choice(n, size=300, replace=False).astype(np.int32)
    g = fl.Graph(w.rowp, w.cols)
    orc = oracle.Graph(w.rowp, w.cols)
    assert np.array_equal(g.ball_sizes(src, 6), orc.ball_sizes(src, 6))
    fac = rng.choice(n, size=2000, replace=False).astype(np.int32)
    cost = np.full(n, np.inf)
    cost[fac] = w.cost[fac]
    g.build_sketches(w.k, w.seed)
    s = fl.Solve(g)
    r = s.compute_radii_exact(cost, w.client)
    assert np.all(np.isinf(np.delete(r, fac)))
    assert np.array_equal(r[fac], orc.exact_radii(cost, w.client, fac))
    s.close()
    g.close()
