#!/usr/bin/env python3
"""Quality report: the GPU path's cost against the oracle's references
(Section 5.2, Table 2 compares the method with a sequential local search).

    python tests/quality_report.py        (needs the GPU library; prints one JSON line)

Enumerable instances (24 ER graphs, 16 vertices): objective / optimum for the
sketch radii with k = 4 and k = 32 (exact sketches at this size) and the
exact-count radii.  Graphs of 1-2 thousand vertices (R-MAT scales 10, 11 with
the workloads' recipe; ER with average degree 10), all vertices clients and
facilities, costs log-uniform [5, 500]: objective / the add/drop/swap local
search from the cheapest facility, and that local search restarted from the
GPU's k = 32 solution.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import flsynth  # noqa: E402
import oracle  # noqa: E402
import paper_1503_03635_gb300 as fl  # noqa: E402

TINY = 24
MAX_MOVES = 5000


def ours(rowp, cols, k, cost, client, exact=False):
    g = fl.Graph(rowp, cols)
    g.build_sketches(k, 1)
    s = fl.Solve(g)
    (s.compute_radii_exact if exact else s.compute_radii)(cost, client)
    op, _ = s.open_facilities()
    s.assign_clients()
    obj = s.objective()[0]
    s.close()
    g.close()
    return op, obj


def main():
    fl.load()
    t0 = time.perf_counter()
    modes = (("k4", 4, False), ("k32", 32, False), ("exact", 32, True))
    tiny = {key: [] for key, _, _ in modes}
    for seed in range(TINY):
        w = flsynth.small_er(16, 2.2, 4000 + seed)
        cost = flsynth.loguniform(16, 4100 + seed, 0.5, 12.0)
        client = flsynth.bernoulli(16, 4200 + seed, 0.85)
        _, opt = oracle.Graph(w.rowp, w.cols).optimum(cost, client)
        for key, k, ex in modes:
            tiny[key].append(ours(w.rowp, w.cols, k, cost, client, ex)[1] / opt)
    table = []
    graphs = [("rmat10", flsynth.rmat(10, 16, 52)), ("rmat11", flsynth.rmat(11, 16, 53))]
    for n in (1000, 2000):
        w = flsynth.small_er(n, 10.0, 54 + n)
        graphs.append((f"er{n}", (w.rowp, w.cols)))
    for name, (rowp, cols) in graphs:
        n = len(rowp) - 1
        cost = flsynth.loguniform(n, 7, 5.0, 500.0)
        client = np.ones(n, np.uint8)
        orc = oracle.Graph(rowp, cols)
        _, ls, moves = orc.local_search(cost, client, max_moves=MAX_MOVES)
        row = {"graph": name, "n": n, "nnz": int(len(cols)), "local_search": ls, "local_search_moves": moves}
        for key, k, ex in modes:
            op, obj = ours(rowp, cols, k, cost, client, ex)
            row[key] = {"objective": obj, "vs_local_search": obj / ls}
            if key == "k32":
                _, ls2, _ = orc.local_search(cost, client, start=op, max_moves=MAX_MOVES)
                row["local_search_from_k32"] = ls2
        table.append(row)
    print(json.dumps({"report": "quality", "seconds": time.perf_counter() - t0,
                      "vs_optimum": {"instances": f"{TINY} ER graphs, n = 16",
                                     **{key: {"mean": float(np.mean(v)), "max": float(np.max(v))}
                                        for key, v in tiny.items()}},
                      "vs_local_search": table}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
