"""A host model of the weighted selection's sweeps, step for step as the
kernels run them (a ring of arrival slots, entry times H - B_f, deadlines,
the two arrival prunings, chunks of steps with jumps over idle stretches),
checked on the CPU against the oracle's sequential greedy and its Dijkstra
assignment.  It shows that the formulation the GPU implements — not only the
kernels, which the GPU tests compare with the oracle — reaches the
lexicographically-first MIS and the nearest-facility assignment, including
on inputs whose greedy takes many rounds and whose ball radii are far above
every distance."""
import math

import numpy as np
import pytest

import brute
import flsynth
import oracle

NONE = 0xFFFFFFFF
CHUNK = 16


def _sweep(rowp, cols, w, R, lab, seeds, H, entry=None, dl=None, dlab=None, first=False, dist=None,
           ft=None, fts=None):
    """Steps 0..H of one sweep; seeds = [(v, value)] entering at time 0."""
    pend = [dict() for _ in range(R)]  # slot -> {vertex: smallest arriving value}

    def arrive(v, x, t):
        if dl is not None and t <= dl[v] and x < dlab[v]:
            dlab[v] = x
        old = lab[v]
        if first:
            if old != NONE:
                return False
            dist[v] = t
        elif x >= old:
            return False
        if ft is not None and old == NONE:
            ft[v] = t
        lab[v] = x
        return True

    front = [v for v, x in seeds if arrive(v, x, 0)]
    t = 0
    while True:
        for _ in range(CHUNK):
            if t > H:
                break
            slot = pend[t % R]
            if t > 0:
                front = []
            for v in sorted(slot):
                if arrive(v, slot[v], t):
                    front.append(v)
            slot.clear()
            if entry is not None and t <= entry["t_last"]:
                for i, f in enumerate(entry["order"]):
                    if entry["B"][f] == H - t and entry["state"][f] == 0 and arrive(f, i, t):
                        front.append(f)
            for u in front:
                x = lab[u]
                for e in range(rowp[u], rowp[u + 1]):
                    v = int(cols[e])
                    if (lab[v] != NONE) if first else (lab[v] <= x):
                        continue
                    t2 = t + int(w[e])
                    if fts is not None and (fts[v] < 0 or t2 > H - fts[v]):
                        continue
                    if t2 > H:
                        continue
                    s2 = pend[t2 % R]
                    s2[v] = min(s2.get(v, NONE), x)
            t += 1
        if t > H:
            break
        if any(pend):
            continue
        if entry is None or t > entry["t_last"]:
            break
        later = [H - entry["B"][f] for f in entry["order"] if entry["B"][f] <= H - t]
        if not later:
            break
        t = max(t, min(later))
        front = []


def _select(rowp, cols, w, r, client, seed):
    n = len(rowp) - 1
    R = int(w.max()) + 1
    order = sorted((f for f in range(n) if math.isfinite(r[f])), key=lambda f: (r[f], oracle.priority(seed, f)))
    B = [-1] * n
    for f in order:
        B[f] = min(int(math.floor(r[f])), 2**31 - 1)
    state = [3] * n
    for f in order:
        state[f] = 0
    rounds = 0
    while True:
        und = [f for f in order if state[f] == 0]
        if not und:
            break
        rounds += 1
        H = max(B[f] for f in und)
        entry = dict(order=order, B=B, state=state, t_last=H - min(B[f] for f in und))
        cover, ft = [NONE] * n, [-1] * n
        _sweep(rowp, cols, w, R, cover, [], H, entry=entry, ft=ft)
        lab, dlab = [NONE] * n, [NONE] * n
        _sweep(rowp, cols, w, R, lab, [(v, cover[v]) for v in range(n) if client[v] and cover[v] != NONE], H,
               dl=B, dlab=dlab, fts=ft)
        joined = 0
        for i, f in enumerate(order):
            if state[f] == 0 and (dlab[f] == NONE or dlab[f] == i):
                state[f] = 1
                joined += 1
            elif state[f] == 0:
                assert dlab[f] < i  # a smaller key shares a client
        claimed = [v for v in range(n) if client[v] and cover[v] != NONE and state[order[cover[v]]] == 1]
        assert joined > 0
        if len(und) > joined and claimed:
            lab, dlab = [NONE] * n, [NONE] * n
            _sweep(rowp, cols, w, R, lab, [(v, v) for v in claimed], H, dl=B, dlab=dlab, fts=ft)
            for f in order:
                if state[f] == 0 and dlab[f] != NONE:
                    state[f] = 2
    return np.array([1 if s == 1 else 0 for s in state], np.uint8), rounds


def _assign(rowp, cols, w, op):
    n = len(rowp) - 1
    lab, dist = [NONE] * n, [-1] * n
    _sweep(rowp, cols, w, int(w.max()) + 1, lab, [(v, v) for v in range(n) if op[v]], 2**31 - 1, first=True,
           dist=dist)
    return np.array([-1 if x == NONE else x for x in lab], np.int32), np.array(dist, np.int32)


def _check(rowp, cols, w, k, seed, cost, client):
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(k, seed)
    r = g.radii(cost, client)
    op, _ = g.open_facilities_weighted(r, client, seed)
    got, rounds = _select(rowp, cols, w, r, client, seed)
    assert np.array_equal(op, got)
    a, d = g.assign_weighted(op)
    a2, d2 = _assign(rowp, cols, w, op)
    assert np.array_equal(a, a2) and np.array_equal(d, d2)
    g.close()
    return rounds


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_model_on_er_with_the_full_length_range(seed):
    wl = flsynth.small_er(250, 4.0, 100 + seed)
    w = flsynth.edge_weights(wl.rowp, wl.cols, seed)
    fac = flsynth.bernoulli(wl.n, seed + 7, 0.5)
    cost = flsynth.loguniform(wl.n, seed + 8, 1.0, 400.0, fac)
    client = flsynth.bernoulli(wl.n, seed + 9, 0.7)
    _check(wl.rowp, wl.cols, w, 8, seed, cost, client)


def test_model_on_rmat_with_narrow_lengths():
    rowp, cols = flsynth.rmat(8, 8, 201)
    n = len(rowp) - 1
    w = flsynth.edge_weights(rowp, cols, 4, 1, 3)
    fac = flsynth.bernoulli(n, 11, 0.6)
    cost = flsynth.loguniform(n, 12, 2.0, 60.0, fac)
    client = flsynth.bernoulli(n, 13, 0.8)
    _check(rowp, cols, w, 16, 4, cost, client)


def test_model_on_a_chain_of_rounds():
    n = 120
    rowp, cols = brute.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    w = np.ones(len(cols), np.int32)
    rounds = _check(rowp, cols, w, 4, 0, np.linspace(2.0, 8.0, n), np.ones(n, np.uint8))
    assert rounds >= 10


def test_model_on_components_with_huge_radii():
    wl = flsynth.small_er(300, 1.2, 87)
    w = flsynth.edge_weights(wl.rowp, wl.cols, 15)
    fac = flsynth.bernoulli(wl.n, 40, 0.15)
    cost = flsynth.loguniform(wl.n, 41, 1.0, 1.0e9, fac)
    client = flsynth.bernoulli(wl.n, 42, 0.5)
    _check(wl.rowp, wl.cols, w, 8, 9, cost, client)
