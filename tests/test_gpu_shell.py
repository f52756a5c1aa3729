"""Reduction by 1-shell (Section "Index Size Reduction"): the index is built
on the graph with its degree-1 trees peeled off, and a tree vertex is
answered through its root. Every answer must equal the oracle's on the whole
graph; the core index must be the oracle's index of the 2-core."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import pspc_inputs as P
from tests import _graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pspc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_00977_gb300 as lib

    lib.load()
    return lib


def two_core(g):
    """Vertices of the 2-core (repeated removal of vertices with at most one
    neighbour left) and the connected components of g."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    deg = g.degree().astype(np.int64)
    alive = np.ones(g.n, bool)
    stack = list(np.flatnonzero(deg <= 1))
    while stack:
        v = stack.pop()
        if not alive[v]:
            continue
        alive[v] = False
        for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            if alive[u]:
                deg[u] -= 1
                if deg[u] <= 1:
                    stack.append(u)
    adj = csr_matrix((np.ones(g.arcs, np.int8), g.col, g.row_ptr), shape=(g.n, g.n))
    _, comp = connected_components(adj, directed=False)
    return alive, comp


def induced(g, rank, keep):
    ids = np.flatnonzero(keep)
    new = -np.ones(g.n, np.int64)
    new[ids] = np.arange(len(ids))
    e = g.edges()
    e = e[keep[e[:, 0]] & keep[e[:, 1]]]
    sub = P.csr_from_edges(len(ids), new[e])
    r = np.argsort(np.argsort(rank[ids], kind="stable"), kind="stable").astype(np.int32)
    return sub, r


def graph_with_trees(seed):
    rng = np.random.default_rng(seed)
    base = G.gnp(40, 0.12, seed)
    e = [tuple(x) for x in base.edges()]
    n = base.n
    for _ in range(30):  # hang random trees off random vertices
        p = int(rng.integers(0, n))
        e.append((p, n))
        n += 1
    for _ in range(3):  # a path component and an isolated edge
        e.append((n, n + 1))
        n += 2
    n += 2  # two isolated vertices
    return P.csr_from_edges(n, np.array(e))


CASES = {
    "path": lambda: (G.path(30), None),
    "star": lambda: (P.csr_from_edges(12, np.array([(0, i) for i in range(1, 12)])), None),
    "tree": lambda: (G.random_tree(80, 7), None),
    "trees_on_gnp": lambda: (graph_with_trees(3), None),
    "ba_m1": lambda: (P.barabasi_albert(300, 1, 5), None),
    "rmat12": lambda: P.workload("rmat12_ef16")[:2],
    "paper": lambda: G.load_paper_table()[:2],
}


@pytest.mark.parametrize("name", list(CASES))
def test_reduced_index_answers_every_pair(pspc, name):
    g, rank = CASES[name]()
    if rank is None:
        rank = P.degree_rank(g, "random", 9)
    rank = np.ascontiguousarray(rank, np.int32)
    full = oracle.OracleIndex(g, rank)
    ix = pspc.Index.from_graph(g, rank, reduce_shell=True)
    try:
        st = ix.stats()
        alive, comp = two_core(g)
        tree_comps = [c for c in np.unique(comp) if not alive[comp == c].any()]
        # peeled: everything but the 2-core and one vertex of each tree component
        assert st["shell_vertices"] == g.n - int(alive.sum()) - len(tree_comps)
        if alive.any():
            sub, r = induced(g, rank, alive)
            core_entries = oracle.OracleIndex(sub, r).entries
        else:
            core_entries = 0
        assert st["entries"] == core_entries + len(tree_comps)  # one isolated core vertex per tree component
        n = g.n
        pairs = np.array([(s, t) for s in range(n) for t in range(n)], np.int32)
        if len(pairs) > 200000:
            pairs = pairs[np.random.default_rng(1).choice(len(pairs), 200000, replace=False)]
        rd, rc, rf, _ = full.query(pairs)
        d, c, f = ix.query(pairs)
        assert np.array_equal(d, rd) and np.array_equal(c, rc) and np.array_equal(f, rf)
    finally:
        ix.free()


def test_reduced_rmat16_matches_full_index(pspc):
    """On R-MAT 16 (42% of the vertices in the 1-shell, most of them isolated)
    the reduced index answers 10^5 pairs like the full GPU index, and stores
    fewer entries."""
    import torch

    g, rank, pairs_fn = P.workload("rmat16")
    pairs = pairs_fn(100000)
    full = pspc.Index.from_graph(g, rank)
    red = pspc.Index.from_graph(g, rank, reduce_shell=True)
    try:
        a = full.query(pairs)
        b = red.query(torch.from_numpy(pairs).cuda())
        assert all(np.array_equal(x, y.cpu().numpy()) for x, y in zip(a, b))
        assert red.stats()["entries"] < full.stats()["entries"]
        assert red.stats()["shell_vertices"] > 0
    finally:
        full.free()
        red.free()


def test_reduced_index_limits(pspc):
    g, rank = G.random_tree(50, 2), None
    rank = P.degree_rank(g, "id")
    ix = pspc.Index.from_graph(g, rank, reduce_shell=True)
    try:
        with pytest.raises(pspc.PSPCError):
            ix.export()
        with pytest.raises(pspc.PSPCError):
            ix.landmarks()
        with pytest.raises(pspc.PSPCError) as e:
            ix.query(np.array([[0, g.n]], np.int32))
        assert e.value.code == 1
    finally:
        ix.free()
