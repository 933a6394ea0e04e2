"""GPU: the serving loop returns, for every query, the plain result of that
query alone, whether it ran alone or batched with others (continuous
batching over two workers with their own streams), and that four of the
results equal the oracle's solve of the query."""
import threading
import time

import numpy as np
import pytest

import flsynth
import oracle
import paper_1503_03635_gb300 as fl
from paper_1503_03635_gb300 import serve

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def test_served_results_equal_plain_results_alone_and_in_the_mix():
    torch = pytest.importorskip("torch")
    rowp, cols = flsynth.rmat(14, 16, 616)
    n = len(rowp) - 1
    k, seed = 16, 9
    g = fl.Graph(rowp, cols)
    g.build_sketches(k, seed)
    srv = serve.Server(g, k, seed, workers=2, max_slots=4)
    sizes = flsynth.loguniform(14, 5, 50.0, 8000.0)
    costs = flsynth.loguniform(14, 6, 10.0, 1000.0)
    qs = [serve.Query(costs[i], client_seed=100 + i, client_frac=sizes[i] / n) for i in range(14)]
    # the first alone, then a burst (batched), then stragglers
    srv.submit(qs[0]).wait(120)
    for q in qs[1:11]:
        srv.submit(q)
    for q in qs[11:]:
        time.sleep(0.01)
        srv.submit(q)
    for q in qs:
        q.wait(120)
    srv.close()
    assert max(q.batch_size for q in qs) > 1 and qs[0].batch_size == 1
    dev = torch.device("cuda", 0)
    og = oracle.Graph(rowp, cols)
    og.build_sketches(k, seed)
    for j, q in enumerate(qs):
        mask = torch.empty(n, dtype=torch.uint8, device=dev)
        serve.client_mask_on_device(torch, n, q.client_seed, q.client_frac, dev, mask)
        s = fl.Solve(g)
        s.compute_radii(np.full(n, q.cost), mask.cpu().numpy())
        op, no = s.open_facilities()
        s.assign_clients()
        obj, ds, un = s.objective()
        s.close()
        assert q.result["n_open"] == no and q.result["dist_sum"] == ds and q.result["n_unserved"] == un
        assert np.array_equal(q.result["open"], op)
        assert abs(q.result["objective"] - obj) <= RTOL * abs(obj)
        if j in (0, 3, 7, 12):
            # the query alone (0), in the burst (3, 7) and a straggler (12)
            # against the oracle
            cl = mask.cpu().numpy()
            cost = np.full(n, q.cost)
            r = og.radii(cost, cl)
            op_w, no_w = og.open_facilities(r, cl, seed)
            _, d_w = og.assign(op_w)
            obj_w, ds_w, un_w = oracle.objective(op_w, cost, cl, d_w)
            assert np.array_equal(q.result["open"], op_w) and q.result["n_open"] == no_w
            assert q.result["dist_sum"] == ds_w and q.result["n_unserved"] == un_w
            assert abs(q.result["objective"] - obj_w) <= RTOL * abs(obj_w)
    og.close()
    g.close()
