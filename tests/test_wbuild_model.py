"""A host model of the weighted ADS build as the kernels run it — entries
(u, v) paired with entries (v, u) of the same length by one sort, levels in
Dijkstra order, a vertex that gains entries marking its neighbours' paired
entries for level L + w, an active vertex merging only its marked entries
through per-entry cursors — checked on the CPU against the oracle's ADS (the
definition, pinned to Floyd-Warshall).  It shows that reading only the marked
entries loses nothing, and that the pairing is a length-preserving
involution that rejects an edge whose lengths differ by direction."""
import bisect

import numpy as np
import pytest

import brute
import flsynth
import oracle


def _pair(rowp, cols, w):
    """rev[e] for every entry, or None when some edge's lengths differ by direction."""
    n = len(rowp) - 1
    src = np.repeat(np.arange(n), np.diff(rowp))
    a = np.minimum(src, cols).astype(np.uint64)
    b = np.maximum(src, cols).astype(np.uint64)
    hi = (a << np.uint64(32)) | b
    lo = (w.astype(np.uint64) << np.uint64(1)) | (src > cols).astype(np.uint64)
    order = np.lexsort((lo, hi))
    H, L, V = hi[order].tolist(), lo[order].tolist(), order.tolist()
    keys = list(zip(H, L))
    rev = [-1] * len(cols)
    for i in range(len(cols)):
        h, l = H[i], L[i]
        if (h >> 32) == (h & 0xFFFFFFFF):
            rev[V[i]] = V[i]
            continue
        l0 = l & ~1
        g0, g1 = bisect.bisect_left(keys, (h, l0)), bisect.bisect_left(keys, (h, l0 + 2))
        half = (g1 - g0) >> 1
        if (g1 - g0) & 1 or half < 1 or L[g0 + half - 1] != l0 or L[g0 + half] != (l0 | 1):
            return None
        if not l & 1:
            rev[V[i]], rev[V[i + half]] = V[i + half], V[i]
    return np.array(rev)


def _build(rowp, cols, w, k, seed):
    """Per vertex the (id, distance) entries of its ADS."""
    n = len(rowp) - 1
    R = int(w.max()) + 1
    rank = [oracle.rank(seed, v) for v in range(n)]
    vertex_of = {r: v for v, r in enumerate(rank)}
    rev = _pair(rowp, cols, w)
    S = [[rank[v]] for v in range(n)]
    rows = [[(v, 0)] for v in range(n)]
    cursor = [0] * len(cols)
    marks = [set() for _ in range(R)]
    active = [set() for _ in range(R)]

    def post(e, level):
        marks[level % R].add(int(rev[e]))
        active[level % R].add(int(cols[e]))

    for e in range(len(cols)):
        post(e, int(w[e]))
    L = 0
    while True:
        nxt = next((L + d for d in range(1, R + 1) if active[(L + d) % R]), None)
        if nxt is None:
            break
        L = nxt
        act, mk = sorted(active[L % R]), marks[L % R]
        active[L % R], marks[L % R] = set(), set()
        have = [len(r) for r in rows]  # row counts as the level starts
        gains = {}
        for v in act:
            cand = set()
            for e in range(rowp[v], rowp[v + 1]):
                if e not in mk:
                    continue
                u, x = int(cols[e]), L - int(w[e])
                c = cursor[e]
                while c < have[u] and rows[u][c][1] < x:
                    c += 1
                c0 = c
                while c < have[u] and rows[u][c][1] == x:
                    c += 1
                cursor[e] = c
                cand.update(rank[rows[u][q][0]] for q in range(c0, c))
            merged = sorted(set(S[v]) | cand)[:k]
            new = sorted(set(merged) - set(S[v]))
            S[v] = merged
            if new:
                gains[v] = new
        for v, new in gains.items():
            rows[v].extend((vertex_of[r], L) for r in new)
            for e in range(rowp[v], rowp[v + 1]):
                post(e, L + int(w[e]))
    return rows


def _oracle_rows(rowp, cols, w, k, seed):
    n = len(rowp) - 1
    g = oracle.Graph(rowp, cols)
    g.set_weights(w)
    g.build_sketches_weighted(k, seed)
    A = g.ads(ranks=False)
    g.close()
    out = []
    for v in range(n):
        e, row = A["eofs"][v], []
        for gi in range(A["gofs"][v], A["gofs"][v + 1]):
            for _ in range(A["gcnt"][gi]):
                row.append((int(A["eid"][e]), int(A["ghop"][gi])))
                e += 1
        out.append(sorted(row))
    return out


def _graph(kind, t):
    if kind == "er":
        wl = flsynth.small_er(200, 4.0, 10 + t)
        return wl.rowp, wl.cols
    if kind == "rmat":
        return flsynth.rmat(8, 8, 20 + t)
    # a path with self-loops and a duplicated edge
    return brute.csr_from_edges(30, [(i, i + 1) for i in range(29)] + [(3, 3), (5, 6), (7, 7)])


@pytest.mark.parametrize("kind,k,hi", [("er", 4, 100), ("rmat", 16, 10), ("odd", 2, 5), ("er", 8, 3)])
def test_marked_entry_build_equals_the_oracle_ads(kind, k, hi):
    rowp, cols = _graph(kind, hi)
    w = flsynth.edge_weights(rowp, cols, hi, 1, hi)
    got = [sorted(r) for r in _build(rowp, cols, w, k, 3)]
    assert got == _oracle_rows(rowp, cols, w, k, 3)


@pytest.mark.parametrize("kind", ["er", "rmat", "odd"])
def test_pairing_is_a_length_preserving_involution(kind):
    rowp, cols = _graph(kind, 1)
    n = len(rowp) - 1
    w = flsynth.edge_weights(rowp, cols, 2, 1, 4)
    rev = _pair(rowp, cols, w)
    src = np.repeat(np.arange(n), np.diff(rowp))
    assert rev is not None
    assert np.array_equal(src[rev], cols) and np.array_equal(cols[rev], src) and np.array_equal(w[rev], w)
    assert np.array_equal(rev[rev], np.arange(len(cols)))
    e = int(np.flatnonzero(src != cols)[0])
    w2 = w.copy()
    w2[e] = w[e] % 4 + 1
    assert _pair(rowp, cols, w2) is None
