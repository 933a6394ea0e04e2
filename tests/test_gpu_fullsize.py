"""GPU parity at full size: the R-MAT scale-26 workload (67,108,864 vertices,
about 2.1e9 CSR entries, k = 16; clients Bernoulli(0.5), facilities
Bernoulli(0.1) with log-uniform costs in [10, 10^4]) in the launch
configuration bench.py times (device-resident inputs on one stream).

The oracle cannot rebuild every sketch at this size, so it checks:
  * sampled vertices' ADS (Algorithm 1 run for the single vertex: ids, hops,
    counted prefixes, HIP weights bit-exact) and their radii (Eq. 1);
  * the radii of 2000 sampled facilities read off the GPU's own ADS rows;
  * the whole open set: that it is the lexicographically-first MIS of the
    conflict graph under the GPU radii (Section 4.3), by its characterisation
    (independent, and every other candidate conflicts with a member of
    smaller key), checked in parallel over facilities;
  * the whole assignment and distances: the oracle's multi-source BFS from
    the GPU open set, plus per-client BFS for sampled clients;
  * the objective, within 1e-9 relative.
Takes a few minutes (workload generation and the CPU passes)."""
import time

import numpy as np
import pytest

import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def _say(t0, what):
    print(f"[{time.perf_counter() - t0:7.1f} s] {what}", flush=True)


def _row(ads, v):
    g0, g1 = ads["gofs"][v], ads["gofs"][v + 1]
    e0, e1 = ads["eofs"][v], ads["eofs"][v + 1]
    return dict(ghop=ads["ghop"][g0:g1], gcnt=ads["gcnt"][g0:g1], gcounted=ads["gcounted"][g0:g1],
                gwt=ads["gwt"][g0:g1], eid=ads["eid"][e0:e1])


def test_rmat26_full_size_sampled_and_global_parity():
    torch = pytest.importorskip("torch")
    t0 = time.perf_counter()
    w = flsynth.config("rmat26")
    _say(t0, f"workload n={w.n} nnz={w.nnz}")

    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(device=dev)
    rowp_d = torch.from_numpy(w.rowp).to(dev)
    cols_d = torch.from_numpy(w.cols).to(dev)
    cost_d = torch.from_numpy(w.cost).to(dev)
    client_d = torch.from_numpy(w.client).to(dev)
    radii_d = torch.empty(w.n, dtype=torch.float64, device=dev)
    open_d = torch.empty(w.n, dtype=torch.uint8, device=dev)
    assign_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    dist_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    g = fl.Graph(rowp_d, cols_d, stream=stream)
    g.build_sketches(w.k, w.seed)
    s = fl.Solve(g)
    s.compute_radii(cost_d, client_d, radii_d)
    _, n_open = s.open_facilities(open_d)
    s.assign_clients(assign_d, dist_d)
    obj, dsum, unserved = s.objective()
    torch.cuda.synchronize()
    ads = g.export_ads()
    s.close()
    g.close()
    radii = radii_d.cpu().numpy()
    op = open_d.cpu().numpy()
    asg = assign_d.cpu().numpy()
    dist = dist_d.cpu().numpy()
    del rowp_d, cols_d, cost_d, client_d, radii_d, open_d, assign_d, dist_d
    _say(t0, f"GPU solve done: {n_open} open, objective {obj}")

    og = oracle.Graph(w.rowp, w.cols)
    deg = np.diff(w.rowp)
    fac = np.flatnonzero(np.isfinite(w.cost) & (deg > 0))
    pick = flsynth.hashes(4, flsynth.QUERY_SEED)

    # sampled vertices: Algorithm 1 for the single vertex, then its radius
    for v in (int(fac[pick[0] % len(fac)]), int(np.argmax(deg))):
        want = og.vertex_ads(w.k, w.seed, v)
        got = _row(ads, v)
        for key in ("ghop", "gcnt", "gcounted"):
            assert np.array_equal(got[key], want[key]), (v, key)
        assert np.array_equal(got["gwt"].view(np.uint64), want["gwt"].view(np.uint64)), v
        assert np.array_equal(got["eid"], want["eid"]), v
        r_want = oracle.radius_of_ads(want, w.client, w.cost[v])
        assert (np.isinf(r_want) and np.isinf(radii[v])) or abs(radii[v] - r_want) <= RTOL * abs(r_want), v
    _say(t0, "sampled single-vertex ADS and radii match")

    # radii of sampled facilities from the GPU's own ADS rows (the radius arithmetic at full size)
    sample = fac[flsynth.hashes(2000, flsynth.QUERY_SEED + 1) % len(fac)]
    for v in sample:
        r_want = oracle.radius_of_ads(_row(ads, v), w.client, w.cost[v])
        assert (np.isinf(r_want) and np.isinf(radii[v])) or abs(radii[v] - r_want) <= RTOL * abs(r_want), v
    del ads
    _say(t0, "2000 sampled radii match")

    # the whole open set: the lexicographically-first MIS on the GPU radii
    ok, bad = og.check_open_facilities(radii, w.client, w.seed, op)
    assert ok, bad
    assert int(op.sum()) == n_open
    _say(t0, "open set is the lexicographically-first MIS")

    # the whole assignment from that open set, and per-client BFS for a sample
    wa, wd = og.assign(op)
    assert np.array_equal(dist, wd)
    assert np.array_equal(asg, wa)
    clients = np.flatnonzero(w.client)
    for c in clients[flsynth.hashes(20, flsynth.QUERY_SEED + 2) % len(clients)]:
        assert og.nearest_open(op, int(c)) == (asg[c], dist[c])
    _say(t0, "assignment matches")

    want_obj, want_ds, want_un = oracle.objective(op, w.cost, w.client, dist)
    assert dsum == want_ds and unserved == want_un
    assert abs(obj - want_obj) <= RTOL * abs(want_obj)
    og.close()
    _say(t0, "objective matches")
