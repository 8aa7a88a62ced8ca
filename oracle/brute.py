"""Betweenness by enumeration of shortest paths -- TEST INFRASTRUCTURE.

Follows the definitions of Section 1.1 word for word, for tiny graphs only:
d(s,t) is the least path length; lambda_st the number of s-t paths of that
length; lambda_st(v) the number of those with v inside; the pair-dependency
delta_st(v) = lambda_st(v)/lambda_st; BC(v) = sum over ordered pairs s != v != t.
Arithmetic is exact (Python ints and fractions.Fraction).

Two enumerators: :func:`all_simple_paths_min` lists every simple path and keeps
the lightest (no distance table at all, n <= 7); :func:`shortest_paths` walks
only extensions that can still be shortest, pruned with Floyd-Warshall
distances (n <= 12 or so).
"""
from __future__ import annotations

from fractions import Fraction

INF = float("inf")


def adjacency(g):
    """Neighbour lists with weights: adj[u] = [(v, w), ...]."""
    adj = [[] for _ in range(g.n)]
    for u in range(g.n):
        for e in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            adj[u].append((int(g.col[e]), 1 if g.w is None else int(g.w[e])))
    return adj


def floyd_warshall(g):
    """All-pairs distances (exact ints, INF when unreachable)."""
    n = g.n
    d = [[INF] * n for _ in range(n)]
    for u, nb in enumerate(adjacency(g)):
        d[u][u] = 0
        for v, w in nb:
            d[u][v] = min(d[u][v], w)
    for k in range(n):
        dk = d[k]
        for i in range(n):
            dik = d[i][k]
            if dik == INF:
                continue
            di = d[i]
            for j in range(n):
                if dik + dk[j] < di[j]:
                    di[j] = dik + dk[j]
    return d


def shortest_paths(g, d=None):
    """Every shortest s-t path (s != t) as a tuple of vertices, keyed by (s, t)."""
    n = g.n
    adj = adjacency(g)
    if d is None:
        d = floyd_warshall(g)
    out = {}
    for s in range(n):
        for t in range(n):
            if s == t or d[s][t] == INF:
                continue
            paths = []
            target = d[s][t]

            def walk(x, length, path):
                if x == t:
                    paths.append(tuple(path))
                    return
                for y, w in adj[x]:
                    if y not in path and length + w + d[y][t] == target:
                        path.append(y)
                        walk(y, length + w, path)
                        path.pop()

            walk(s, 0, [s])
            out[(s, t)] = paths
    return out


def all_simple_paths_min(g):
    """Shortest paths with no distance table: enumerate every simple s-t path
    and keep those of least total weight."""
    n = g.n
    adj = adjacency(g)
    out = {}
    for s in range(n):
        found = {}

        def walk(x, length, path):
            if x != s:
                found.setdefault(x, []).append((length, tuple(path)))
            for y, w in adj[x]:
                if y not in path:
                    path.append(y)
                    walk(y, length + w, path)
                    path.pop()

        walk(s, 0, [s])
        for t, lst in found.items():
            best = min(L for L, _ in lst)
            out[(s, t)] = [p for L, p in lst if L == best]
    return out


def betweenness(g, paths=None, sources=None):
    """Exact results from the path sets: dict with bc (list of Fraction,
    ordered pairs), dist (n x n, None unreachable), lam (n x n ints, lam[s][s]=1),
    dep (n x n Fractions, dep[s][v] = delta_s*(v), v != s)."""
    n = g.n
    if paths is None:
        paths = shortest_paths(g)
    src = range(n) if sources is None else sources
    bc = [Fraction(0)] * n
    dist = [[None] * n for _ in range(n)]
    lam = [[0] * n for _ in range(n)]
    dep = [[Fraction(0)] * n for _ in range(n)]
    wts = {}
    for u, nb in enumerate(adjacency(g)):
        for v, w in nb:
            wts[(u, v)] = w
    for s in range(n):
        dist[s][s] = 0
        lam[s][s] = 1
    for (s, t), ps in paths.items():
        lam[s][t] = len(ps)
        dist[s][t] = sum(wts[(ps[0][i], ps[0][i + 1])] for i in range(len(ps[0]) - 1))
    for s in src:
        for t in range(n):
            if t == s or (s, t) not in paths:
                continue
            ps = paths[(s, t)]
            through = [0] * n
            for p in ps:
                for v in p[1:-1]:
                    through[v] += 1
            for v in range(n):
                if through[v]:
                    f = Fraction(through[v], len(ps))
                    dep[s][v] += f
                    bc[v] += f
    return dict(bc=bc, dist=dist, lam=lam, dep=dep)
