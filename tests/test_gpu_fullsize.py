"""GPU parity at full size, element by element against the oracle's own full
build, in the launch configuration bench.py times (device-resident inputs on
one stream):

  * the R-MAT scale-26 workload (67,108,864 vertices, about 2.1e9 CSR
    entries, k = 16; clients Bernoulli(0.5), facilities Bernoulli(0.1) with
    log-uniform costs in [10, 10^4]);
  * the serving workload's resident graph (R-MAT scale 23, k = 32) with one
    query's client set and cost, solved plainly.

Compared: hop count and edge-merges; every sketch (ranks and counts); the
whole ADS (offsets, group hops, counts, counted prefixes, the bit patterns
of the HIP weights, entry ids); every radius (Eq. 1) against the oracle's
radii from its own ADS, within 1e-9 relative; the open set against the
oracle's characterisation of the lexicographically-first MIS under the
oracle's radii (Section 4.3: independent, and every other candidate
conflicts with a member of smaller key); the whole assignment and distances
against the oracle's multi-source BFS from that open set; the objective.
Two vertices' ADS are also rebuilt by Algorithm 1 for the single vertex.

Host memory: about 125 GB at the peak of the scale-26 oracle build (the
workload, the GPU's exported sketches and ADS, and the oracle's build
state).  Takes several minutes, mostly the oracle's build on the host
cores."""
import gc
import time

import numpy as np
import pytest

import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu

RTOL = 1e-9
ADS_KEYS = ("gofs", "eofs", "ghop", "gcnt", "gcounted", "eid")


def _say(t0, what):
    print(f"[{time.perf_counter() - t0:7.1f} s] {what}", flush=True)


def _row(ads, v):
    g0, g1 = ads["gofs"][v], ads["gofs"][v + 1]
    e0, e1 = ads["eofs"][v], ads["eofs"][v + 1]
    return dict(ghop=ads["ghop"][g0:g1], gcnt=ads["gcnt"][g0:g1], gcounted=ads["gcounted"][g0:g1],
                gwt=ads["gwt"][g0:g1], eid=ads["eid"][e0:e1])


def _first_diff(a, b):
    d = np.flatnonzero(a != b)
    return None if len(d) == 0 else (int(d[0]), a[d[0]], b[d[0]], len(d))


def _gpu_solve(w, t0):
    """The whole path on the GPU from device-resident inputs; every output
    and the sketches and ADS exported to host memory."""
    import torch

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
    out = dict(stats=g.stats(), n_open=n_open, objective=obj, dist_sum=dsum, n_unserved=unserved)
    _say(t0, f"GPU solve done: {n_open} open, objective {obj}, {out['stats']}")
    out["S"], out["Scnt"] = g.export_sketches()
    out["ads"] = g.export_ads()
    s.close()
    g.close()
    out["radii"] = radii_d.cpu().numpy()
    out["open"] = open_d.cpu().numpy()
    out["assign"] = assign_d.cpu().numpy()
    out["dist"] = dist_d.cpu().numpy()
    del rowp_d, cols_d, cost_d, client_d, radii_d, open_d, assign_d, dist_d
    torch.cuda.empty_cache()
    _say(t0, "GPU outputs exported")
    return out


def _compare_with_full_oracle(w, got, t0, alg1_vertices=()):
    og = oracle.Graph(w.rowp, w.cols)
    og.build_sketches(w.k, w.seed)
    _say(t0, f"oracle build done on {oracle.threads()} threads: {og.hops} hops, {og.edge_merges} edge-merges")
    assert got["stats"]["hops"] == og.hops
    assert got["stats"]["edge_merges"] == og.edge_merges

    # every sketch
    S, cnt = og.sketch()
    assert np.array_equal(got["Scnt"], cnt), _first_diff(got["Scnt"], cnt)
    assert np.array_equal(got["S"], S), _first_diff(got["S"].ravel(), S.ravel())
    del S, cnt
    got.pop("S"), got.pop("Scnt")
    gc.collect()
    _say(t0, "every sketch matches")

    # the whole ADS
    want = og.ads(ranks=False)
    ads = got["ads"]
    assert got["stats"]["ads_entries"] == len(want["eid"])
    assert got["stats"]["ads_groups"] == len(want["ghop"])
    for key in ADS_KEYS:
        assert np.array_equal(ads[key], want[key]), (key, _first_diff(ads[key], want[key]))
    assert np.array_equal(ads["gwt"].view(np.uint64), want["gwt"].view(np.uint64)), \
        ("gwt", _first_diff(ads["gwt"].view(np.uint64), want["gwt"].view(np.uint64)))
    del want
    gc.collect()
    _say(t0, f"the whole ADS matches ({got['stats']['ads_entries']} entries)")

    # Algorithm 1 for single vertices (the oracle's hop-synchronous build
    # against the sequential definition, at full size)
    for v in alg1_vertices:
        want = og.vertex_ads(w.k, w.seed, int(v))
        row = _row(ads, int(v))
        for key in ("ghop", "gcnt", "gcounted", "eid"):
            assert np.array_equal(row[key], want[key]), (v, key)
        assert np.array_equal(row["gwt"].view(np.uint64), want["gwt"].view(np.uint64)), v
    got.pop("ads")
    del ads
    gc.collect()

    # every radius, from the oracle's own ADS
    r_want = og.radii(w.cost, w.client)
    r = got["radii"]
    inf_w, inf_g = np.isinf(r_want), np.isinf(r)
    assert np.array_equal(inf_w, inf_g), _first_diff(inf_w, inf_g)
    fin = ~inf_w
    rel = np.abs(r[fin] - r_want[fin]) / np.abs(r_want[fin])
    assert rel.size == 0 or rel.max() <= RTOL, (rel.max(), int(np.argmax(rel)))
    _say(t0, f"{int(fin.sum())} finite radii match (max rel {rel.max() if rel.size else 0:.3g}, "
             f"{int((r[fin] == r_want[fin]).sum())} bit-identical)")

    # the open set: the lexicographically-first MIS under the oracle's radii
    op = got["open"]
    ok, bad = og.check_open_facilities(r_want, w.client, w.seed, op)
    assert ok, bad
    assert int(op.sum()) == got["n_open"]
    _say(t0, "open set is the lexicographically-first MIS under the oracle's radii")

    # the whole assignment and distances
    wa, wd = og.assign(op)
    assert np.array_equal(got["dist"], wd), _first_diff(got["dist"], wd)
    assert np.array_equal(got["assign"], wa), _first_diff(got["assign"], wa)
    _say(t0, "assignment and distances match")

    want_obj, want_ds, want_un = oracle.objective(op, w.cost, w.client, wd)
    assert got["dist_sum"] == want_ds and got["n_unserved"] == want_un
    assert abs(got["objective"] - want_obj) <= RTOL * abs(want_obj)
    og.close()
    _say(t0, "objective matches")


def test_rmat26_full_size_parity_with_the_full_oracle_build():
    pytest.importorskip("torch")
    t0 = time.perf_counter()
    w = flsynth.config("rmat26")
    _say(t0, f"workload n={w.n} nnz={w.nnz}")
    got = _gpu_solve(w, t0)
    deg = np.diff(w.rowp)
    fac = np.flatnonzero(np.isfinite(w.cost) & (deg > 0))
    v0 = int(fac[flsynth.hashes(1, flsynth.QUERY_SEED)[0] % len(fac)])
    _compare_with_full_oracle(w, got, t0, alg1_vertices=(v0, int(np.argmax(deg))))


def test_serving_graph_rmat23_k32_plain_solve_parity():
    """The serving workload's resident graph (R-MAT scale 23, edge factor 16,
    the same recipe as the serving benchmark, k = 32) with one query: clients
    Bernoulli(m/n) with m = 10^5, every vertex a facility at cost 100."""
    pytest.importorskip("torch")
    t0 = time.perf_counter()
    rowp, cols = flsynth.rmat(23, 16, 42 + 5)
    n = len(rowp) - 1
    client = flsynth.bernoulli(n, flsynth.QUERY_SEED + 7, 1.0e5 / n)
    w = flsynth.from_csr("rmat23", rowp, cols, 32, flsynth.SKETCH_SEED, np.full(n, 100.0), client)
    _say(t0, f"workload n={w.n} nnz={w.nnz} clients={int(client.sum())}")
    got = _gpu_solve(w, t0)
    _compare_with_full_oracle(w, got, t0, alg1_vertices=(int(np.argmax(np.diff(rowp))),))
