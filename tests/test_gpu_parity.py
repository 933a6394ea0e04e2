"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact: sketches, ADS (ids, hops, counted flags, HIP weights), hop and
edge-merge counts, open sets, assignments and distances.  Floating point:
radii and objective within 1e-9 relative (the kernels use the oracle's
operation order, so radii are in practice bit-identical).
"""
import numpy as np
import pytest

import brute
import flsynth
import oracle
import paper_1503_03635_gb300 as fl

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def _gpu(w):
    g = fl.Graph(w.rowp, w.cols)
    g.build_sketches(w.k, w.seed)
    S, cnt = g.export_sketches()
    ads = g.export_ads()
    st = g.stats()
    s = fl.Solve(g)
    r = s.compute_radii(w.cost, w.client)
    op, nopen = s.open_facilities()
    a, d = s.assign_clients()
    obj, ds, un = s.objective()
    out = dict(S=S, Scnt=cnt, ads=ads, hops=st["hops"], edge_merges=st["edge_merges"], radii=r, open=op,
               n_open=nopen, assign=a, dist=d, objective=obj, dist_sum=ds, n_unserved=un, mis=s.stats())
    s.close()
    g.close()
    return out


def _compare(w, gpu, orc, check_ads=True):
    assert gpu["hops"] == orc["hops"]
    assert gpu["edge_merges"] == orc["edge_merges"]
    assert (gpu["Scnt"] == orc["Scnt"]).all()
    assert (gpu["S"] == orc["S"]).all()
    if check_ads:
        A, B = gpu["ads"], orc["ads"]
        for key in ("gofs", "eofs", "ghop", "gcnt", "gcounted", "eid"):
            assert np.array_equal(A[key], B[key]), key
        # HIP weights: bit-exact (one IEEE division of the same operands)
        assert np.array_equal(A["gwt"].view(np.uint64), B["gwt"].view(np.uint64))
    r1, r2 = gpu["radii"], orc["radii"]
    fin = np.isfinite(r2)
    assert np.array_equal(np.isfinite(r1), fin)
    assert np.all(np.abs(r1[fin] - r2[fin]) <= RTOL * np.abs(r2[fin]))
    assert gpu["n_open"] == orc["n_open"]
    assert np.array_equal(gpu["open"], orc["open"])
    assert np.array_equal(gpu["dist"], orc["dist"])
    assert np.array_equal(gpu["assign"], orc["assign"])
    assert gpu["dist_sum"] == orc["dist_sum"] and gpu["n_unserved"] == orc["n_unserved"]
    assert abs(gpu["objective"] - orc["objective"]) <= RTOL * abs(orc["objective"])


def _oracle(w):
    return oracle.solve(w.rowp, w.cols, w.k, w.seed, w.cost, w.client)


# ------------------------------------------------------------------ tiny graphs

def _tiny(name):
    if name == "path":
        return brute.csr_from_edges(12, [(i, i + 1) for i in range(11)])
    if name == "star":
        return brute.csr_from_edges(9, [(0, i) for i in range(1, 9)])
    if name == "cycle":
        return brute.csr_from_edges(13, [(i, (i + 1) % 13) for i in range(13)])
    if name == "complete":
        return brute.csr_from_edges(7, [(i, j) for i in range(7) for j in range(i + 1, 7)])
    if name == "mixed":
        return brute.csr_from_edges(10, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (4, 6), (8, 9)])
    raise KeyError(name)


@pytest.mark.parametrize("name", ["path", "star", "cycle", "complete", "mixed"])
@pytest.mark.parametrize("k", [2, 4, 16, 32])
def test_tiny_graphs(name, k):
    rowp, cols = _tiny(name)
    n = len(rowp) - 1
    client = (np.arange(n) % 3 != 2).astype(np.uint8)
    cost = np.array([1.5 + 2.0 * (v % 4) for v in range(n)], float)
    cost[n // 2] = np.inf
    w = flsynth.from_csr(name, rowp, cols, k, 7, cost, client)
    _compare(w, _gpu(w), _oracle(w))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_small_er_random_subsets(seed):
    w = flsynth.small_er(300, 3.0, 100 + seed, k=4, cost=6.0, client_p=0.6, fac_p=0.4)
    w.cost = np.where(np.isfinite(w.cost), flsynth.loguniform(w.n, seed, 2.0, 40.0), np.inf)
    _compare(w, _gpu(w), _oracle(w))


def test_er10k_workload():
    """Erdos-Renyi n=10^4, avg degree 8, k=16, uniform cost 20 (first workload)."""
    w = flsynth.config("er10k")
    _compare(w, _gpu(w), _oracle(w))


@pytest.mark.parametrize("scale,k", [(12, 32), (14, 16), (15, 32)])
def test_rmat_several_tiles(scale, k):
    """R-MAT with hubs (warp merges of long rows, many flush rounds), ragged
    frontiers and isolated vertices; clients/facilities as random subsets."""
    rowp, cols = flsynth.rmat(scale, 16, 500 + scale)
    n = len(rowp) - 1
    client = flsynth.bernoulli(n, 3, 0.5)
    fac = flsynth.bernoulli(n, 4, 0.3)
    cost = flsynth.loguniform(n, 5, 10.0, 1.0e4, fac)
    w = flsynth.from_csr(f"rmat{scale}", rowp, cols, k, 1, cost, client)
    _compare(w, _gpu(w), _oracle(w))


def test_rmat20_workload_full():
    """R-MAT scale 20, k=32, all vertices clients and facilities, costs
    log-uniform in [5, 500] (second workload), compared element by element."""
    w = flsynth.config("rmat20")
    _compare(w, _gpu(w), _oracle(w))


def test_hubs_in_push_and_pull_rounds():
    """Two hubs of several kSeg-edge segments each (degrees 6000 and 3000)
    sharing leaves, a long path hanging off them and a few isolated vertices:
    the BFS and the MIS sweeps push hub segments while the frontier is small
    and pull them once it is large."""
    n = 9000
    edges = [(0, i) for i in range(1, 6001)]
    edges += [(6001, i) for i in range(3500, 6500)]
    edges += [(i, i + 1) for i in range(6500, 8990)]
    rowp, cols = brute.csr_from_edges(n, edges)
    client = flsynth.bernoulli(n, 21, 0.7)
    fac = flsynth.bernoulli(n, 22, 0.2)
    fac[[0, 6001, 8500]] = 1
    cost = flsynth.loguniform(n, 23, 3.0, 3000.0, fac)
    for k in (4, 16):
        w = flsynth.from_csr("twohubs", rowp, cols, k, 5, cost, client)
        _compare(w, _gpu(w), _oracle(w))


@pytest.mark.parametrize("scale,k", [(12, 4), (15, 16)])
def test_hop_stats_account_for_every_ads_group(scale, k):
    """Per-hop counters: every (vertex, hop >= 1) ADS group is one changed
    sketch, so n + sum(changed) = ADS groups; the mask merge reads a subset of
    the scanned CSR entries and takes over once sketches fill with small ranks."""
    rowp, cols = flsynth.rmat(scale, 16, 700 + scale)
    n = len(rowp) - 1
    g = fl.Graph(rowp, cols)
    g.profile(True, census=True)
    g.build_sketches(k, 3)
    st = g.stats()
    hs = g.hop_stats()
    g.close()
    assert len(hs) == st["hops"] + 1 and hs[-1]["changed"] == 0
    assert n + sum(h["changed"] for h in hs) == st["ads_groups"]
    assert all(0 <= h["mask"] <= h["scanned"] for h in hs)
    assert hs[0]["mask"] == 0 and hs[0]["scanned"] == len(cols)
    assert sum(h["mask"] for h in hs) > 0
    assert all(h["ms"] > 0 for h in hs)


# ------------------------------------------------------------------ edge cases

def test_single_vertex():
    rowp = np.array([0, 0], np.int64)
    cols = np.zeros(0, np.int32)
    w = flsynth.from_csr("one", rowp, cols, 16, 1, np.array([3.0]), np.array([1], np.uint8))
    gpu, orc = _gpu(w), _oracle(w)
    _compare(w, gpu, orc)
    assert gpu["radii"][0] == 3.0 and gpu["n_open"] == 1 and gpu["objective"] == 3.0


def test_no_edges_no_clients_no_facilities():
    n = 50
    rowp = np.zeros(n + 1, np.int64)
    cols = np.zeros(0, np.int32)
    for cost, client in ((np.full(n, 4.0), np.zeros(n, np.uint8)),
                         (np.full(n, np.inf), np.ones(n, np.uint8))):
        w = flsynth.from_csr("empty", rowp, cols, 8, 1, cost, client)
        gpu, orc = _gpu(w), _oracle(w)
        _compare(w, gpu, orc)
        assert gpu["n_open"] == 0


def test_duplicates_and_self_loops_tolerated():
    # raw CSR with a duplicate edge and self-loops (still symmetric)
    rows = {0: [0, 1, 1, 2], 1: [0, 0, 2], 2: [0, 1, 2, 3], 3: [2]}
    rowp = np.zeros(5, np.int64)
    cols = []
    for v in range(4):
        cols += rows[v]
        rowp[v + 1] = len(cols)
    w = flsynth.from_csr("dups", rowp, np.array(cols, np.int32), 2, 3, np.full(4, 2.5),
                         np.ones(4, np.uint8))
    _compare(w, _gpu(w), _oracle(w))


def test_invalid_csr_and_costs_are_rejected():
    rowp = np.array([0, 1, 2], np.int64)
    with pytest.raises(fl.FLError) as e:
        fl.Graph(rowp, np.array([1, 5], np.int32))  # id out of range
    assert e.value.status == fl.FL_EINVAL
    with pytest.raises(fl.FLError):
        fl.Graph(np.array([0, 2, 1], np.int64), np.array([1, 0], np.int32))  # offsets decrease
    g = fl.Graph(rowp, np.array([1, 0], np.int32))
    with pytest.raises(fl.FLError) as e:
        g.build_sketches(64, 1)
    assert e.value.status == fl.FL_EINVAL
    with pytest.raises(fl.FLError) as e:
        fl.Solve(g)
    assert e.value.status == fl.FL_ESTATE
    g.build_sketches(4, 1)
    s = fl.Solve(g)
    with pytest.raises(fl.FLError) as e:
        s.open_facilities()
    assert e.value.status == fl.FL_ESTATE
    for bad in (np.array([0.0, 1.0]), np.array([-1.0, 1.0]), np.array([np.nan, 1.0])):
        with pytest.raises(fl.FLError) as e:
            s.compute_radii(bad, np.ones(2, np.uint8))
        assert e.value.status == fl.FL_EINVAL
    g.build_sketches(4, 2)  # rebuild invalidates the old solve
    with pytest.raises(fl.FLError) as e:
        s.compute_radii(np.ones(2), np.ones(2, np.uint8))
    assert e.value.status == fl.FL_ESTATE


def test_device_memory_arguments():
    """Inputs and outputs in device memory (torch tensors) give the same results."""
    torch = pytest.importorskip("torch")
    w = flsynth.config("er10k")
    dev = torch.device("cuda:0")
    g = fl.Graph(torch.from_numpy(w.rowp).to(dev), torch.from_numpy(w.cols).to(dev),
                 stream=torch.cuda.current_stream())
    g.build_sketches(w.k, w.seed)
    s = fl.Solve(g)
    r = torch.empty(w.n, dtype=torch.float64, device=dev)
    s.compute_radii(torch.from_numpy(w.cost).to(dev), torch.from_numpy(w.client).to(dev), r)
    op = torch.empty(w.n, dtype=torch.uint8, device=dev)
    _, nopen = s.open_facilities(op)
    a = torch.empty(w.n, dtype=torch.int32, device=dev)
    d = torch.empty(w.n, dtype=torch.int32, device=dev)
    s.assign_clients(a, d)
    orc = _oracle(w)
    assert np.array_equal(r.cpu().numpy(), orc["radii"])
    assert np.array_equal(op.cpu().numpy(), orc["open"]) and nopen == orc["n_open"]
    assert np.array_equal(a.cpu().numpy(), orc["assign"])
    assert np.array_equal(d.cpu().numpy(), orc["dist"])


# ------------------------------------------------------------------ hop model

def _model_from_ads(rowp, cols, ads, hops):
    """Per-hop terms of the algorithmic-bytes model, recomputed from the
    oracle's ADS: |D_h(u)| is the entry count of u's group at hop h."""
    n = len(rowp) - 1
    deg = np.diff(rowp)
    H = hops + 1
    dcnt = np.zeros((H + 1, n), np.int64)
    owner = np.repeat(np.arange(n), np.diff(ads["gofs"]))
    dcnt[ads["ghop"], owner] = ads["gcnt"]
    src = np.repeat(np.arange(n), deg)
    out = []
    for h in range(1, H + 1):
        prev = dcnt[h - 1]
        in_front = prev[cols] > 0
        E = int(in_front.sum())
        A = int(np.unique(src[in_front]).size)
        SD = int((deg * prev).sum())
        out.append(dict(edge_merges=E, merging=A, delta_sum=SD, new_entries=int(dcnt[h].sum())))
    return out


@pytest.mark.parametrize("name", ["er10k", "rmat12"])
def test_hop_model_terms_match_the_oracle_ads(name):
    if name == "er10k":
        w = flsynth.config("er10k")
    else:
        rowp, cols = flsynth.rmat(12, 16, 45)
        n = len(rowp) - 1
        w = flsynth.from_csr("rmat12", rowp, cols, 16, 1, np.full(n, 30.0), np.ones(n, np.uint8))
    og = oracle.Graph(w.rowp, w.cols)
    og.build_sketches(w.k, w.seed)
    want = _model_from_ads(w.rowp, w.cols, og.ads(ranks=False), og.hops)
    g = fl.Graph(w.rowp, w.cols)
    g.build_sketches(w.k, w.seed)
    got = g.hop_model()
    assert len(got) == len(want) == og.hops + 1
    for h, (a, b) in enumerate(zip(got, want)):
        for key in ("edge_merges", "merging", "delta_sum", "new_entries"):
            assert a[key] == b[key], (h + 1, key, a[key], b[key])
        assert a["delta_read"] >= 0
    assert sum(m["edge_merges"] for m in got) == og.edge_merges
    g.close()
    og.close()


def test_long_balls_without_gather_pruning():
    """Ball radii above 254 (a 700-vertex path, costs 1e5): the MIS runs its
    gather sweeps without the per-vertex pruning (its reach counters are one
    byte), and still matches the oracle."""
    n = 700
    rowp, cols = brute.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    client = np.ones(n, np.uint8)
    cost = np.full(n, np.inf)
    cost[[0, 350, 699]] = [1.0e5, 1.0e5, 3.0e4]
    w = flsynth.from_csr("longpath", rowp, cols, 32, 3, cost, client)
    gpu = _gpu(w)
    _compare(w, gpu, _oracle(w))
    assert np.nanmax(np.where(np.isfinite(gpu["radii"]), gpu["radii"], np.nan)) >= 255


@pytest.mark.parametrize("name", ["rmat12", "er10k"])
def test_mis_log_accounts_for_every_candidate(name):
    """fl_mis_log: one total row per greedy round; the bucket sizes of a
    round add up to its undecided facilities, the rounds decide every
    candidate, and each round's undecided count is the previous one's minus
    what it decided."""
    if name == "rmat12":
        rowp, cols = flsynth.rmat(12, 16, 512)
        n = len(rowp) - 1
        w = flsynth.from_csr(name, rowp, cols, 16, 1, flsynth.loguniform(n, 5, 10.0, 1.0e4, flsynth.bernoulli(n, 4, 0.3)),
                             flsynth.bernoulli(n, 3, 0.5))
    else:
        w = flsynth.config(name)
    g = fl.Graph(w.rowp, w.cols)
    g.build_sketches(w.k, w.seed)
    s = fl.Solve(g)
    s.compute_radii(w.cost, w.client)
    s.open_facilities()
    st = s.stats()
    log = s.mis_log()
    s.close()
    g.close()
    assert log.shape[1] == 6
    tot = log[log[:, 1] == 3]
    assert len(tot) == st["mis_rounds"]
    assert list(tot[:, 0]) == list(range(1, st["mis_rounds"] + 1))
    assert tot[0, 3] == st["candidates"]
    assert tot[:, 4].sum() == st["candidates"]
    for i, row in enumerate(tot):
        b = log[(log[:, 0] == row[0]) & (log[:, 1] == 2)]
        assert b[:, 3].sum() == row[3]
        assert b[:, 2].max() == row[2]
        if i + 1 < len(tot):
            assert tot[i + 1, 3] == row[3] - row[4]
    rounds = log[np.isin(log[:, 1], [0, 1])]
    assert np.all(rounds[:, 3] > 0) and np.all(np.isin(rounds[:, 4], [0, 1]))
