"""Brute-force SPC labels and queries with exact (arbitrary-precision) counts.

TEST INFRASTRUCTURE ONLY (see the package docstring). Pure Python; meant
for graphs of at most a few hundred vertices.

Labels follow the ESPC construction by trough shortest paths (Section "PSPC
algorithm description from the Covering Side"): for every pair w, v with w
ranked at or above v, L(v) holds (w, sd(v,w), |C_{v,w}|) when the set
C_{v,w} of trough shortest v-w paths (w ranked above every other vertex of
the path) is non-empty. |C_{v,w}| is obtained as the shortest-path count
from w inside the subgraph induced by w and the vertices ranked below it,
taken only where that restricted distance equals the true distance.

Queries are plain breadth-first shortest-path counting from s, which is what
the ESPC property (Definition "Exact Shortest Path Covering") says the
index must reproduce.
"""
from __future__ import annotations

from collections import deque


def adjacency(n: int, edges) -> list[list[int]]:
    adj: list[set[int]] = [set() for _ in range(n)]
    for u, v in edges:
        u, v = int(u), int(v)
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    return [sorted(a) for a in adj]


def bfs_paths(adj, s: int, allowed=None):
    """(dist, count) dicts of shortest paths from s, exact ints. If
    ``allowed`` is given, only s and vertices in it are traversed."""
    dist = {s: 0}
    cnt = {s: 1}
    q = deque([s])
    while q:
        x = q.popleft()
        for y in adj[x]:
            if allowed is not None and y not in allowed:
                continue
            if y not in dist:
                dist[y] = dist[x] + 1
                cnt[y] = cnt[x]
                q.append(y)
            elif dist[y] == dist[x] + 1:
                cnt[y] += cnt[x]
    return dist, cnt


def labels(n: int, edges, rank) -> list[list[tuple[int, int, int]]]:
    """L(v) as lists of (hub vertex id, dist, exact count), sorted by hub rank."""
    adj = adjacency(n, edges)
    rank = [int(r) for r in rank]
    true = [bfs_paths(adj, s)[0] for s in range(n)]
    L: list[list[tuple[int, int, int]]] = [[] for _ in range(n)]
    for w in sorted(range(n), key=lambda v: rank[v]):
        below = {x for x in range(n) if rank[x] > rank[w]}
        d, c = bfs_paths(adj, w, below)
        for v, dv in d.items():
            if dv == true[w].get(v):
                L[v].append((w, dv, c[v]))
    return L


def spc(n: int, edges, s: int, t: int):
    """(sd(s,t), number of shortest s-t paths) by breadth-first counting;
    (None, 0) when t is unreachable."""
    adj = adjacency(n, edges)
    d, c = bfs_paths(adj, s)
    if t not in d:
        return None, 0
    return d[t], c[t]


def spc_all(n: int, edges):
    """All-pairs (dist, count) tables from breadth-first counting."""
    adj = adjacency(n, edges)
    return [bfs_paths(adj, s) for s in range(n)]
