"""Betweenness centrality straight from its definition, in exact rationals.

    BC(v) = sum over sources s in S (s != v) and targets t reachable from s
            (t != s, t != v) of  sigma_st(v) / sigma_st

where sigma_st counts shortest s-t paths and sigma_st(v) those through v
(Brandes' definition, cited by the paper's Section 2).  Ordered pairs, no
halving.  Distances come from Floyd-Warshall and every shortest path is listed
explicitly, so nothing here shares a step with the Brandes recurrences.
Only for graphs of a dozen vertices or so.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

INF = 1 << 30


def adjacency(g):
    return [list(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]) for v in range(g.n)]


def all_pairs_dist(g):
    n = g.n
    d = [[INF] * n for _ in range(n)]
    for v in range(n):
        d[v][v] = 0
    for v, nb in enumerate(adjacency(g)):
        for w in nb:
            d[v][w] = min(d[v][w], 1)
    for k in range(n):
        dk = d[k]
        for i in range(n):
            dik = d[i][k]
            if dik >= INF:
                continue
            di = d[i]
            for j in range(n):
                if dik + dk[j] < di[j]:
                    di[j] = dik + dk[j]
    return d


def shortest_paths(adj, d, s, t):
    """Every shortest s-t path as a tuple of vertices."""
    out = []

    def walk(path):
        x = path[-1]
        if x == t:
            out.append(tuple(path))
            return
        for y in adj[x]:
            if d[s][y] == len(path) and d[y][t] == d[s][t] - len(path):
                path.append(y)
                walk(path)
                path.pop()

    walk([s])
    return out


def bc_exact(g, sources):
    adj = adjacency(g)
    d = all_pairs_dist(g)
    bc = [Fraction(0)] * g.n
    for s in sources:
        for t in range(g.n):
            if t == s or d[s][t] >= INF:
                continue
            paths = shortest_paths(adj, d, s, t)
            total = len(paths)
            for p in paths:
                for v in p[1:-1]:
                    bc[v] += Fraction(1, total)
    return bc


def sigma_exact(g, s):
    """Number of shortest paths from s to every vertex (0 when unreachable)."""
    adj = adjacency(g)
    d = all_pairs_dist(g)
    return [len(shortest_paths(adj, d, s, t)) if d[s][t] < INF else 0 for t in range(g.n)]


def bfs_dist(g, s):
    """Textbook FIFO BFS with a deque (hop distance, -1 when unreachable)."""
    dist = [-1] * g.n
    dist[s] = 0
    q = deque([s])
    rp, ci = g.row_ptr, g.col_idx
    while q:
        u = q.popleft()
        for e in range(rp[u], rp[u + 1]):
            v = int(ci[e])
            if dist[v] < 0:
                dist[v] = dist[u] + 1
                q.append(v)
    return dist


def pair_distance_excess(g, sources):
    """sum over s in S, t reachable, t != s of (d(s,t) - 1): the total of all BC values."""
    import numpy as np

    total = 0
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    ci = np.asarray(g.col_idx, dtype=np.int64)
    for s in sources:
        dist = np.full(g.n, -1, np.int64)
        dist[s] = 0
        frontier = np.array([s], np.int64)
        level = 0
        while frontier.size:
            starts, ends = rp[frontier], rp[frontier + 1]
            counts = ends - starts
            if counts.sum() == 0:
                break
            idx = np.repeat(starts - np.cumsum(np.concatenate([[0], counts[:-1]])), counts) + np.arange(counts.sum())
            nb = np.unique(ci[idx])
            nb = nb[dist[nb] < 0]
            level += 1
            dist[nb] = level
            frontier = nb
        reached = dist[dist > 0]
        total += int((reached - 1).sum())
    return total


def bc_exact_weighted(g, weights, sources):
    """BC from its definition under positive arc weights (parallel to col_idx):
    weighted Floyd-Warshall distances, every shortest path listed."""
    n = g.n
    rp, ci = g.row_ptr, g.col_idx
    d = [[INF] * n for _ in range(n)]
    wt = {}
    for v in range(n):
        d[v][v] = 0
        for e in range(rp[v], rp[v + 1]):
            x, w = int(ci[e]), int(weights[e])
            d[v][x] = min(d[v][x], w)
            wt.setdefault((v, x), []).append(w)
    for k in range(n):
        for i in range(n):
            if d[i][k] >= INF:
                continue
            for j in range(n):
                if d[i][k] + d[k][j] < d[i][j]:
                    d[i][j] = d[i][k] + d[k][j]
    adj = [[(int(ci[e]), int(weights[e])) for e in range(rp[v], rp[v + 1])] for v in range(n)]
    bc = [Fraction(0)] * n
    for s in sources:
        for t in range(n):
            if t == s or d[s][t] >= INF:
                continue
            paths = []

            def walk(path, dist):
                x = path[-1]
                if x == t:
                    paths.append(tuple(path))
                    return
                for y, w in adj[x]:  # parallel arcs are separate paths
                    if dist + w == d[s][y] and d[s][y] + d[y][t] == d[s][t]:
                        path.append(y)
                        walk(path, dist + w)
                        path.pop()

            walk([s], 0)
            for p in paths:
                for v in p[1:-1]:
                    bc[v] += Fraction(1, len(paths))
    return bc
