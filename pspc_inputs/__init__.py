"""Seeded synthetic inputs for the SPC hub-label build and query.

This module holds the graph and query generators that both the CUDA path
and the CPU oracle are fed from. It contains none of the labelling or query
arithmetic: only graph construction (Barabasi-Albert, R-MAT, perturbed
grid), symmetrisation into CSR, the vertex orders the labelling takes as
input (degree-descending, and the paper's hybrid order of a degree-ordered
core above a tree-decomposition-ordered fringe), and uniform query pairs.

Graphs are undirected and unweighted, as in the paper's problem statement
(Section "Preliminaries", Graphs); directed samples are symmetrised, as the
paper does for its directed datasets (Section "Experimental Settings").

Every generator takes an explicit integer seed and uses numpy's PCG64, so a
(generator, parameters, seed) triple names one graph on every machine.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Graph",
    "barabasi_albert",
    "rmat",
    "perturbed_grid",
    "csr_from_edges",
    "degree_rank",
    "query_pairs",
    "largest_component",
    "workload",
    "ba_batch",
    "elimination_order",
    "hybrid_rank",
]


class Graph:
    """Undirected graph in symmetric CSR form.

    ``row_ptr`` is int64[n+1]; ``col`` is int32[2m] with each row sorted
    ascending, no self-loops and no duplicate arcs; every edge {u,v} is
    stored as both arcs u->v and v->u.
    """

    def __init__(self, n: int, row_ptr: np.ndarray, col: np.ndarray, name: str = ""):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.name = name

    @property
    def arcs(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.arcs // 2

    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edges(self) -> np.ndarray:
        """Edge list [m, 2] with u < v."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degree())
        dst = self.col.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)

    def __repr__(self) -> str:
        return f"Graph({self.name!r}, n={self.n}, m={self.m})"


def csr_from_edges(n: int, edges: np.ndarray, name: str = "") -> Graph:
    """Symmetrise an edge list, drop self-loops and duplicates, build CSR."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if e.size and (e.min() < 0 or e.max() >= n):
        raise ValueError("edge endpoint out of range")
    e = e[e[:, 0] != e[:, 1]]
    src = np.concatenate([e[:, 0], e[:, 1]])
    dst = np.concatenate([e[:, 1], e[:, 0]])
    key = np.unique(src * np.int64(n) + dst)
    src = key // n
    dst = key % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return Graph(n, row_ptr, dst.astype(np.int32), name)


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    """Barabasi-Albert preferential attachment.

    Starts from ``m`` isolated seed vertices 0..m-1. Vertex ``m`` links to all
    of them; every later vertex links to ``m`` distinct earlier vertices
    drawn with probability proportional to their current degree (sampling
    from the list of edge endpoints, rejecting repeats).
    """
    if m < 1 or n <= m:
        raise ValueError("need 1 <= m < n")
    rng = np.random.default_rng(seed)
    ends = np.empty(2 * m * (n - m), dtype=np.int64)  # every edge endpoint so far
    fill = 0
    src = np.empty(m * (n - m), dtype=np.int64)
    dst = np.empty(m * (n - m), dtype=np.int64)
    k = 0
    targets = list(range(m))
    buf = rng.random(4096)
    bi = 0
    for v in range(m, n):
        for t in targets:
            src[k] = v
            dst[k] = t
            k += 1
        ends[fill:fill + m] = targets
        ends[fill + m:fill + 2 * m] = v
        fill += 2 * m
        if v == n - 1:
            break
        chosen: list[int] = []
        seen = set()
        while len(chosen) < m:
            if bi == buf.size:
                buf = rng.random(4096)
                bi = 0
            t = int(ends[int(buf[bi] * fill)])
            bi += 1
            if t not in seen:
                seen.add(t)
                chosen.append(t)
        targets = chosen
    return csr_from_edges(n, np.stack([src[:k], dst[:k]], axis=1), f"ba_n{n}_m{m}_s{seed}")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, d: float,
         seed: int) -> Graph:
    """R-MAT sample of ``edge_factor * 2**scale`` arcs, then symmetrised.

    Each arc picks one quadrant per bit level with probabilities (a, b, c, d):
    a = (0,0), b = (0,1), c = (1,0), d = (1,1). Self-loops and duplicates
    are removed; isolated vertices are kept, so n = 2**scale.
    """
    if abs(a + b + c + d - 1.0) > 1e-9:
        raise ValueError("R-MAT probabilities must sum to 1")
    n = 1 << scale
    ne = edge_factor * n
    rng = np.random.default_rng(seed)
    src = np.zeros(ne, dtype=np.int64)
    dst = np.zeros(ne, dtype=np.int64)
    for bit in range(scale):
        r = rng.random(ne)
        sbit = r >= (a + b)
        dbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        src |= sbit.astype(np.int64) << bit
        dst |= dbit.astype(np.int64) << bit
    return csr_from_edges(n, np.stack([src, dst], axis=1), f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def largest_component(g: Graph) -> Graph:
    """Largest connected component, relabelled compactly in increasing id."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    adj = csr_matrix((np.ones(g.arcs, dtype=np.int8), g.col, g.row_ptr), shape=(g.n, g.n))
    ncomp, lab = connected_components(adj, directed=False)
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    newid = -np.ones(g.n, dtype=np.int64)
    newid[keep] = np.arange(keep.size)
    e = g.edges()
    e = e[(newid[e[:, 0]] >= 0) & (newid[e[:, 1]] >= 0)]
    return csr_from_edges(keep.size, newid[e], g.name + "_lcc")


def perturbed_grid(k: int, delete_frac: float, seed: int) -> Graph:
    """k x k 4-neighbour grid with floor(delete_frac * E) edges deleted
    uniformly at random, reduced to its largest connected component."""
    ids = np.arange(k * k, dtype=np.int64).reshape(k, k)
    horiz = np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], axis=1)
    vert = np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], axis=1)
    e = np.concatenate([horiz, vert])
    rng = np.random.default_rng(seed)
    ndel = int(np.floor(delete_frac * len(e)))
    drop = rng.choice(len(e), size=ndel, replace=False)
    keep = np.ones(len(e), dtype=bool)
    keep[drop] = False
    g = csr_from_edges(k * k, e[keep], f"grid{k}_del{delete_frac}_s{seed}")
    return largest_component(g)


def degree_rank(g: Graph, tie: str = "id", seed: int | None = None) -> np.ndarray:
    """Degree-descending vertex order as a rank array (0 = highest rank).

    Ties are broken by vertex id (``tie='id'``) or by a seeded random
    permutation (``tie='random'``). Returns int32 rank[v] in [0, n).
    """
    deg = g.degree()
    if tie == "id":
        tiekey = np.arange(g.n)
    elif tie == "random":
        tiekey = np.random.default_rng(seed).permutation(g.n)
    else:
        raise ValueError(tie)
    order = np.lexsort((tiekey, -deg))
    rank = np.empty(g.n, dtype=np.int32)
    rank[order] = np.arange(g.n, dtype=np.int32)
    return rank


def elimination_order(g: Graph, delta: int | None = None):
    """Minimum-degree elimination (the tree-decomposition order of the
    paper's Section "Vertex Order", road network order): repeatedly remove
    a vertex of smallest current degree (ties by vertex id) and join its
    remaining neighbours pairwise (fill edges), so the degrees of the
    neighbours become their true degrees in the reduced graph.

    With ``delta`` given, elimination stops as soon as every remaining
    vertex has more than ``delta`` neighbours. Returns (eliminated vertex
    ids in elimination order, remaining vertex ids ascending, degree of
    every vertex in the reduced graph at the stop, 0 for eliminated ones)."""
    import heapq

    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    heap = [(len(adj[v]), v) for v in range(g.n)]
    heapq.heapify(heap)
    gone = np.zeros(g.n, dtype=bool)
    order = []
    while heap:
        dv, v = heapq.heappop(heap)
        if gone[v] or dv != len(adj[v]):
            continue  # stale entry
        if delta is not None and dv > delta:
            break
        gone[v] = True
        order.append(v)
        nb = list(adj[v])
        for x in nb:
            adj[x].discard(v)
        for i, x in enumerate(nb):
            for y in nb[i + 1:]:
                if y not in adj[x]:
                    adj[x].add(y)
                    adj[y].add(x)
        for x in nb:
            heapq.heappush(heap, (len(adj[x]), x))
        adj[v] = set()
    rest = np.flatnonzero(~gone)
    reduced = np.array([len(a) for a in adj], dtype=np.int64)
    return np.asarray(order, dtype=np.int64), rest, reduced


def hybrid_rank(g: Graph, delta: int | None = 5) -> np.ndarray:
    """Hybrid vertex order (Section "Vertex Order", Hybrid Vertex Ordering),
    as a rank array (0 = highest). The fringe is what minimum-degree
    elimination removes while some vertex has at most ``delta`` neighbours
    in the reduced graph; the rest is the core. Core vertices rank above
    all fringe vertices, by degree descending in the reduced graph (the
    core with its fill edges; ties by degree in G, then by id); fringe
    vertices follow in reverse elimination order (the last one removed
    ranks highest), the tree-decomposition order. ``delta=None``
    eliminates every vertex: the pure tree-decomposition order."""
    fringe, core, reduced = elimination_order(g, delta)
    deg = g.degree()
    core = core[np.lexsort((core, -deg[core], -reduced[core]))]
    order = np.concatenate([core, fringe[::-1]])
    rank = np.empty(g.n, dtype=np.int32)
    rank[order] = np.arange(g.n, dtype=np.int32)
    return rank


def query_pairs(n: int, q: int, seed: int) -> np.ndarray:
    """int32[q, 2] of uniform (s, t) pairs; s == t is allowed."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, size=(q, 2), dtype=np.int64).astype(np.int32)


def _ba_member(args):
    i, n, m, seed = args
    g = barabasi_albert(int(n), int(m), int(seed))
    return i, g.n, g.row_ptr, g.col, degree_rank(g, "id")


def ba_batch(count: int = 512, n_range=(500, 20000), m_range=(2, 8), seed: int = 1000, workers: int = 0):
    """A batch of Barabasi-Albert graphs of uneven size: graph i has
    n_i ~ U[n_range] and m_i ~ U{m_range} (both drawn with numpy seed
    ``seed``), is generated with seed ``seed + i``, and is ranked by degree
    descending (ties by id). Returns a list of (n, row_ptr, col, rank).
    ``workers`` > 1 generates in a spawn process pool."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=count)
    ms = np.minimum(ms, ns - 1)
    jobs = [(i, ns[i], ms[i], seed + i) for i in range(count)]
    out = [None] * count
    if workers and workers > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(workers) as pool:
            for i, n, rp, col, rank in pool.imap_unordered(_ba_member, jobs, chunksize=4):
                out[i] = (n, rp, col, rank)
    else:
        for job in jobs:
            i, n, rp, col, rank = _ba_member(job)
            out[i] = (n, rp, col, rank)
    return out


RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def workload(name: str):
    """Named workloads: returns (graph, rank, pairs_fn) where pairs_fn(q)
    draws q query pairs with the workload's pair seed.

    * ``ba2000``: Barabasi-Albert n=2,000, m=4, seed 1, ties by id.
    * ``rmat16``: R-MAT scale 16, edge factor 16, (0.57,0.19,0.19,0.05),
      seed 1, ties by id; pairs seed 2.
    * ``rmat20``: R-MAT scale 20, edge factor 8, same parameters, seed 1,
      random ties with seed 3; pairs seed 2.
    * ``grid256``: 256x256 grid, 10% of edges deleted, seed 1, largest
      component, random ties with seed 3; pairs seed 2.

    A suffix ``@hybrid<delta>`` or ``@td`` replaces the degree order by the
    hybrid order with that threshold or by the pure tree-decomposition
    order (``hybrid_rank``), e.g. ``grid256@td``.
    """
    if "@" in name:
        base, how = name.split("@", 1)
        g, _, pf = workload(base)
        if how == "td":
            return g, hybrid_rank(g, None), pf
        if how.startswith("hybrid") and how[6:].isdigit():
            return g, hybrid_rank(g, int(how[6:])), pf
        raise KeyError(name)
    if name == "ba2000":
        g = barabasi_albert(2000, 4, 1)
        rank = degree_rank(g, "id")
    elif name == "rmat16":
        g = rmat(16, 16, *RMAT_ABCD, seed=1)
        rank = degree_rank(g, "id")
    elif name == "rmat20":
        g = rmat(20, 8, *RMAT_ABCD, seed=1)
        rank = degree_rank(g, "random", 3)
    elif name == "grid256":
        g = perturbed_grid(256, 0.10, 1)
        rank = degree_rank(g, "random", 3)
    elif name.startswith("rmat") and "_ef" in name:
        # rmat<scale>_ef<edge_factor>: smaller R-MAT graphs of the same family
        sc, ef = name[4:].split("_ef")
        g = rmat(int(sc), int(ef), *RMAT_ABCD, seed=1)
        rank = degree_rank(g, "id")
    elif name.startswith("grid") and name[4:].isdigit():
        g = perturbed_grid(int(name[4:]), 0.10, 1)
        rank = degree_rank(g, "random", 3)
    else:
        raise KeyError(name)
    return g, rank, (lambda q, _n=g.n: query_pairs(_n, q, 2))
