"""Brute-force definitions for tiny graphs (test helpers, pure Python).

Everything here is computed from first principles on a materialised
all-pairs distance table, independently of the oracle's propagation code:

* balls and bottom-k sketches of balls (Section 3.3: the ADS is the union of
  the min-hash sketches of the l closest vertices, for every l);
* the ADS by definition, with HIP weights from the definition of the
  conditional inclusion probability (Cohen 2014, cited in Section 3.3);
* the exact root of the epsilon->0 opening condition (Eq. 1) from exact
  client distances, in rational arithmetic;
* the conflict graph H-bar (Algorithm 3) and its lexicographically-first MIS;
* nearest-open-facility assignment and the objective (Section 3.1).
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np

TWO64 = float(2 ** 64)


def csr_from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    rowp = np.zeros(n + 1, np.int64)
    cols = []
    for v in range(n):
        nb = sorted(adj[v])
        cols.extend(nb)
        rowp[v + 1] = rowp[v] + len(nb)
    return rowp, np.array(cols, np.int32)


def adjacency(rowp, cols):
    n = len(rowp) - 1
    return [list(cols[rowp[v]:rowp[v + 1]]) for v in range(n)]


def apsp(rowp, cols) -> np.ndarray:
    """All-pairs hop distances by one BFS per vertex; -1 = unreachable."""
    adj = adjacency(rowp, cols)
    n = len(adj)
    D = np.full((n, n), -1, np.int64)
    for s in range(n):
        D[s, s] = 0
        q = deque([s])
        while q:
            x = q.popleft()
            for u in adj[x]:
                if D[s, u] < 0:
                    D[s, u] = D[s, x] + 1
                    q.append(u)
    return D


def apsp_weighted(rowp, cols, w) -> np.ndarray:
    """All-pairs distances with edge lengths w (one per CSR entry) by
    Floyd-Warshall; -1 = unreachable."""
    n = len(rowp) - 1
    INF = 1 << 60
    D = [[INF] * n for _ in range(n)]
    for v in range(n):
        D[v][v] = 0
        for e in range(int(rowp[v]), int(rowp[v + 1])):
            u = int(cols[e])
            D[v][u] = min(D[v][u], int(w[e]))
    for m in range(n):
        Dm = D[m]
        for i in range(n):
            dim = D[i][m]
            if dim >= INF:
                continue
            Di = D[i]
            for j in range(n):
                if dim + Dm[j] < Di[j]:
                    Di[j] = dim + Dm[j]
    out = np.array(D, np.int64)
    out[out >= INF] = -1
    return out


def ball(D, v, h):
    return [w for w in range(D.shape[0]) if 0 <= D[v, w] <= h]


def bottom_k(values, k):
    return sorted(values)[:k]


def sketch_at(D, rk, k, v, h):
    """S_h(v): the k smallest ranks of the ball of radius h around v."""
    return bottom_k([int(rk[w]) for w in ball(D, v, h)], k)


def max_ecc(D):
    return int(D.max()) if D.size else 0


def ads_by_definition(D, rk, k):
    """ADS(v) = {(w, d(v,w)) : r(w) is among the k smallest ranks of the ball
    of radius d(v,w)}; each entry carries `counted` (it is among the k-1
    smallest, or the ball has fewer than k vertices) and its HIP weight:
    1 / Pr[w counted | all other ranks] = 2^64 / t, where t is the (k-1)-th
    smallest rank of the ball without w (weight 1 when that ball has fewer
    than k-1 vertices).  Returned per vertex as a list of
    (hop, sorted [(rank, id, counted, weight)])."""
    n = D.shape[0]
    out = []
    for v in range(n):
        groups = []
        hmax = int(D[v].max())
        for h in range(hmax + 1):
            B = ball(D, v, h)
            ranks_B = sorted(int(rk[w]) for w in B)
            entries = []
            for w in B:
                if D[v, w] != h:
                    continue
                r = int(rk[w])
                if r not in ranks_B[:k]:
                    continue
                others = sorted(int(rk[x]) for x in B if x != w)
                counted = len(ranks_B) < k or r in ranks_B[:k - 1]
                if len(others) < k - 1:
                    wt = 1.0
                else:
                    wt = TWO64 / float(others[k - 2])
                entries.append((r, w, counted, wt))
            if entries:
                groups.append((h, sorted(entries)))
        out.append(groups)
    return out


def exact_radius(dists, cost):
    """Root r >= 0 of sum_c max(0, r - d_c) = cost (exact, Fraction)."""
    ds = sorted(int(d) for d in dists)
    if not ds:
        return None
    cost = Fraction(cost)
    # on [ds[i], ds[i+1]] the slope is i+1 and g(ds[i]) = sum_{j<i} (ds[i]-ds[j])
    for i in range(len(ds)):
        g_i = sum(Fraction(ds[i] - ds[j]) for j in range(i))
        hi = ds[i + 1] if i + 1 < len(ds) else None
        g_hi = None if hi is None else g_i + (i + 1) * (hi - ds[i])
        if hi is None or g_hi >= cost:
            return ds[i] + (cost - g_i) / (i + 1)
    return None


def conflict_graph(D, r, client):
    """H-bar on candidates (finite r): f ~ g iff some client is within
    floor(r_f) of f and within floor(r_g) of g."""
    n = D.shape[0]
    cand = [f for f in range(n) if np.isfinite(r[f])]
    balls = {}
    for f in cand:
        B = int(np.floor(r[f]))
        balls[f] = {c for c in range(n) if client[c] and 0 <= D[f, c] <= B}
    adj = {f: set() for f in cand}
    for i, f in enumerate(cand):
        for g in cand[i + 1:]:
            if balls[f] & balls[g]:
                adj[f].add(g)
                adj[g].add(f)
    return cand, balls, adj


def lfmis(cand, adj, key):
    """Lexicographically-first MIS: scan in key order, take f unless a
    neighbour was already taken."""
    S = set()
    for f in sorted(cand, key=key):
        if not (adj[f] & S):
            S.add(f)
    return S


def nearest_assignment(D, open_set):
    n = D.shape[0]
    a = np.full(n, -1, np.int64)
    d = np.full(n, -1, np.int64)
    for v in range(n):
        best = None
        for f in sorted(open_set):
            if D[v, f] >= 0 and (best is None or D[v, f] < best):
                best = D[v, f]
                a[v] = f
        if best is not None:
            d[v] = best
    return a, d


# ---------------------------------------------------------------- epsilon > 0
# The opening phase of Algorithms 3-5 and the selection of Algorithm 6 on an
# all-pairs distance table (exact client counts instead of ADS estimates),
# written from the paper's text with the readings listed in the oracle:
# alpha_0 = gamma (1 + eps) / m^2, alpha_j = alpha_{j-1} (1 + eps); a client
# at distance delta counts in the shell of the smallest grid value >= delta;
# q(f) sums (1 + eps) alpha(c) - d_c over clients whose shell value d_c is at
# most alpha(c); facilities open before clients freeze, within one iteration.

def eps_gamma(D, cost, client) -> float:
    """max over clients with a reachable facility of min_f (c(f) + d(c, f)); -1 if none."""
    n = D.shape[0]
    best = -1.0
    for c in range(n):
        if not client[c]:
            continue
        vals = [cost[f] + float(D[c, f]) for f in range(n) if np.isfinite(cost[f]) and D[c, f] >= 0]
        if vals:
            best = max(best, min(vals))
    return best


def eps_opening(D, cost, client, eps):
    n = D.shape[0]
    onepe = 1.0 + eps
    fac = [f for f in range(n) if np.isfinite(cost[f])]
    cli = [c for c in range(n) if client[c]]
    fac_iter = np.full(n, -1, np.int64)
    cli_iter = np.full(n, -1, np.int64)
    q = np.zeros(n)
    if not fac or not cli:
        return dict(fac_iter=fac_iter, cli_iter=cli_iter, q=q, alpha0=0.0, iterations=0)
    gamma = eps_gamma(D, cost, client)
    if gamma < 0:
        return dict(fac_iter=fac_iter, cli_iter=cli_iter, q=q, alpha0=0.0, iterations=0)
    m = float(len(fac)) * float(len(cli))
    alpha0 = (gamma * onepe) / (m * m)
    grid = [alpha0]

    def alpha(j):
        while len(grid) <= j:
            grid.append(grid[-1] * onepe)
        return grid[j]

    def shell(delta):
        j = 0
        while alpha(j) < delta:
            j += 1
        return j

    reach = [c for c in cli if any(D[c, f] >= 0 for f in fac)]
    unfrozen = set(reach)
    unopened = set(fac)
    j = 0
    while unopened and unfrozen:
        j += 1
        new = []
        for f in sorted(unopened):
            total = 0.0
            for c in cli:
                if D[f, c] < 0:
                    continue
                jc = cli_iter[c] if cli_iter[c] >= 0 else j
                sc = shell(D[f, c])
                if sc <= jc:
                    total += onepe * alpha(jc) - alpha(sc)
            q[f] = total
            if total >= cost[f]:
                new.append(f)
        for f in new:
            fac_iter[f] = j
            unopened.discard(f)
        opened = [f for f in range(n) if fac_iter[f] >= 0]
        for c in sorted(unfrozen):
            d = min((D[c, f] for f in opened if D[c, f] >= 0), default=-1)
            if d >= 0 and float(d) <= onepe * alpha(j):
                cli_iter[c] = j
                unfrozen.discard(c)
    return dict(fac_iter=fac_iter, cli_iter=cli_iter, q=q, alpha0=alpha0, iterations=j)


def eps_hbar(D, eps, alpha0, fac_iter, cli_iter):
    """H-bar of Algorithm 6: open facilities f_a, f_b conflict iff a client
    c with alpha(c) = alpha(f_a) = alpha(f_b) is within (1 + eps) alpha(c)
    of both."""
    n = D.shape[0]
    onepe = 1.0 + eps
    grid = [alpha0]
    for _ in range(int(max(fac_iter.max(), 0))):
        grid.append(grid[-1] * onepe)
    opened = [f for f in range(n) if fac_iter[f] >= 0]
    wit = {}
    for f in opened:
        j = int(fac_iter[f])
        wit[f] = {c for c in range(n) if cli_iter[c] == j and 0 <= D[f, c] and float(D[f, c]) <= onepe * grid[j]}
    adj = {f: {g for g in opened if g != f and wit[f] & wit[g]} for f in opened}
    return opened, adj
