"""Small graphs with closed-form shortest-path counts, shared by the oracle
and GPU tests. Only graph construction lives here: no labelling or query
arithmetic."""
from __future__ import annotations

import itertools
import re
from math import comb, factorial

import numpy as np

from pspc_inputs import Graph, csr_from_edges, degree_rank

GOLDEN_DIR = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def path(n: int) -> Graph:
    return csr_from_edges(n, np.array([(i, i + 1) for i in range(n - 1)]).reshape(-1, 2), f"path{n}")


def cycle(n: int) -> Graph:
    return csr_from_edges(n, np.array([(i, (i + 1) % n) for i in range(n)]), f"cycle{n}")


def complete(n: int) -> Graph:
    return csr_from_edges(n, np.array(list(itertools.combinations(range(n), 2))), f"K{n}")


def grid(k: int) -> Graph:
    """k x k 4-neighbour grid, vertex r*k + c."""
    e = []
    for r in range(k):
        for c in range(k):
            v = r * k + c
            if c + 1 < k:
                e.append((v, v + 1))
            if r + 1 < k:
                e.append((v, v + k))
    return csr_from_edges(k * k, np.array(e), f"grid{k}")


def bipartite_2m(m: int) -> Graph:
    """K(2, m): middle vertices 0..m-1, each joined to s = m and t = m + 1.
    SPC(s, t) = (2, m); two middle vertices are at distance 2 with 2 paths."""
    e = [(w, m) for w in range(m)] + [(w, m + 1) for w in range(m)]
    return csr_from_edges(m + 2, np.array(e), f"K2,{m}")


def hub_ladder(m: int, depth: int) -> Graph:
    """m hubs 0..m-1, each joined to both vertices of layer 1 of a ladder of
    width 2 and the given depth (vertices m + 2(k-1), m + 2(k-1) + 1 in
    layer k; consecutive layers completely joined). A hub reaches a layer-k
    vertex by 2^(k-1) shortest paths of length k."""
    e = [(z, m + i) for z in range(m) for i in range(2)]
    for k in range(1, depth):
        a, b = m + 2 * (k - 1), m + 2 * k
        e += [(a + i, b + j) for i in range(2) for j in range(2)]
    return csr_from_edges(m + 2 * depth, np.array(e), f"hubladder{m}x{depth}")


def hypercube(k: int) -> Graph:
    n = 1 << k
    e = [(v, v ^ (1 << b)) for v in range(n) for b in range(k) if v < v ^ (1 << b)]
    return csr_from_edges(n, np.array(e), f"Q{k}")


def diamond_chain(k: int) -> Graph:
    """k diamonds in series: a_i -> {b_i, c_i} -> a_{i+1}; a_i = 3i,
    b_i = 3i+1, c_i = 3i+2, a_k = 3k. 2^k shortest a_0 - a_k paths."""
    e = []
    for i in range(k):
        a, b, c, a2 = 3 * i, 3 * i + 1, 3 * i + 2, 3 * (i + 1)
        e += [(a, b), (a, c), (b, a2), (c, a2)]
    return csr_from_edges(3 * k + 1, np.array(e), f"diamonds{k}")


def random_tree(n: int, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    e = [(v, int(rng.integers(0, v))) for v in range(1, n)]
    return csr_from_edges(n, np.array(e).reshape(-1, 2), f"tree{n}")


def gnp(n: int, p: float, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return csr_from_edges(n, np.stack([iu[0][keep], iu[1][keep]], 1), f"gnp{n}_{p}_{seed}")


def random_rank(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).permutation(n).astype(np.int32)


def closed_forms():
    """(graph, s, t, sd, exact count) cases with textbook answers."""
    cases = []
    g = path(9)
    cases.append((g, 0, 8, 8, 1))
    g = cycle(10)
    cases.append((g, 0, 5, 5, 2))
    cases.append((g, 2, 5, 3, 1))
    g = cycle(11)
    cases.append((g, 0, 5, 5, 1))
    g = complete(7)
    cases.append((g, 1, 6, 1, 1))
    for k in (4, 6):
        g = grid(k)
        cases.append((g, 0, k * k - 1, 2 * k - 2, comb(2 * k - 2, k - 1)))
    for k in (3, 4, 5):
        g = hypercube(k)
        cases.append((g, 0, (1 << k) - 1, k, factorial(k)))
    for k in (5, 63, 64, 65):
        g = diamond_chain(k)
        cases.append((g, 0, 3 * k, 2 * k, 2 ** k))
    return cases


def load_paper_table():
    """The paper's 10-vertex example: (graph, rank, table, example) with
    0-based ids; table[v] = list of (hub, dist, count)."""
    import os

    txt = open(os.path.join(GOLDEN_DIR, "paper_table_labels.txt")).read()
    order = [int(x) - 1 for x in re.search(r"^order: (.*)$", txt, re.M).group(1).split()]
    edges = [tuple(int(y) - 1 for y in e.split("-"))
             for e in re.search(r"^edges: (.*)$", txt, re.M).group(1).split()]
    ex = [int(x) for x in re.search(r"^example: (.*)$", txt, re.M).group(1).split()]
    table = {}
    for m in re.finditer(r"^L (\d+): (.*)$", txt, re.M):
        table[int(m.group(1)) - 1] = [(int(h) - 1, int(d), int(c)) for h, d, c in
                                      re.findall(r"\((\d+),(\d+),(\d+)\)", m.group(2))]
    n = 10
    rank = np.empty(n, np.int32)
    rank[order] = np.arange(n, dtype=np.int32)
    g = csr_from_edges(n, np.array(edges), "paper_fig1")
    example = (ex[0] - 1, ex[1] - 1, ex[2], ex[3])
    return g, rank, table, example


__all__ = ["path", "cycle", "complete", "grid", "hypercube", "diamond_chain", "random_tree",
           "gnp", "random_rank", "closed_forms", "load_paper_table", "degree_rank"]
