"""Vertex orders of the paper's Section "Vertex Order": minimum-degree
elimination (the tree-decomposition order) and the hybrid order of a
degree-ordered core above a tree-decomposition-ordered fringe. The labels
are defined for any order, so the oracle is pinned under these orders too."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import brute
import pspc_inputs as P
from tests import _graphs as G


def replay_min_degree(g, order, delta):
    """Dense-matrix replay of an elimination sequence: at each step the
    vertex removed has the smallest degree among the remaining ones (ties by
    id) and at most ``delta`` neighbours; its neighbours are joined. Returns
    the reduced adjacency after the last step."""
    A = np.zeros((g.n, g.n), dtype=bool)
    for v in range(g.n):
        A[v, g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] = True
    alive = np.ones(g.n, dtype=bool)
    for v in order:
        deg = A[alive][:, alive].sum(axis=1)
        ids = np.flatnonzero(alive)
        best = ids[np.lexsort((ids, deg))[0]]
        assert v == best, (v, best)
        nb = np.flatnonzero(A[v] & alive)
        assert delta is None or len(nb) <= delta
        A[np.ix_(nb, nb)] = True
        A[nb, nb] = False
        A[v, :] = False
        A[:, v] = False
        alive[v] = False
    return A, alive


@pytest.mark.parametrize("case", ["tree", "cycle", "complete", "grid", "gnp", "ba"])
@pytest.mark.parametrize("delta", [1, 2, 3, 5, None])
def test_elimination_is_min_degree_with_fill(case, delta):
    g = {"tree": lambda: G.random_tree(60, 3), "cycle": lambda: G.cycle(30), "complete": lambda: G.complete(8),
         "grid": lambda: G.grid(7), "gnp": lambda: G.gnp(50, 0.1, 4),
         "ba": lambda: P.barabasi_albert(80, 2, 5)}[case]()
    order, rest, reduced = P.elimination_order(g, delta)
    A, alive = replay_min_degree(g, order, delta)
    assert sorted(order.tolist() + rest.tolist()) == list(range(g.n))
    assert np.array_equal(np.flatnonzero(alive), rest)
    sub = A[np.ix_(rest, rest)].sum(axis=1)
    assert np.array_equal(reduced[rest], sub)
    if delta is not None and len(rest):
        assert sub.min() > delta  # stopped only when every vertex has more than delta neighbours
    if case == "tree" and delta is not None:
        assert len(rest) == 0  # a tree always has a leaf
    if case == "cycle":
        assert len(rest) == (g.n if delta == 1 else 0)
    if case == "complete":
        assert len(rest) == (0 if delta is None or delta >= 7 else g.n)


def test_hybrid_rank_layout():
    g = P.perturbed_grid(12, 0.1, 3)
    for delta in (2, 3, 5, None):
        rank = P.hybrid_rank(g, delta)
        assert sorted(rank.tolist()) == list(range(g.n))
        fringe, core, reduced = P.elimination_order(g, delta)
        assert np.all(rank[core] < len(core))  # core above the fringe
        assert np.array_equal(rank[fringe[::-1]], np.arange(len(core), g.n))  # reverse elimination order
        key = [(-int(reduced[v]), -int(g.degree()[v]), int(v)) for v in core]
        assert [int(v) for v in core[np.argsort(rank[core])]] == [v for _, _, v in sorted(key)]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("delta", [2, 5, None])
def test_oracle_under_hybrid_orders_matches_definition(seed, delta):
    g = G.gnp(14, 0.25, 100 + seed) if seed % 2 else P.perturbed_grid(4, 0.1, seed)
    rank = P.hybrid_rank(g, delta)
    want = brute.labels(g.n, g.edges().tolist(), rank)
    got = oracle.OracleIndex(g, rank).export()
    for v in range(g.n):
        lab = [(int(got.hub[i]), int(got.dist[i]) & 0x7FFF, int(got.cnt[i])) for i in range(got.off[v], got.off[v + 1])]
        assert lab == [(h, d, c % (1 << 64)) for h, d, c in want[v]], v


def test_td_order_shrinks_grid_labels():
    """The paper motivates the tree-decomposition order by road-like
    graphs: on a perturbed grid its index is several times smaller than the
    degree order's (for this 48x48 grid, about a third)."""
    g, rank, _ = P.workload("grid48")
    deg = oracle.OracleIndex(g, rank).entries
    td = oracle.OracleIndex(g, P.hybrid_rank(g, None)).entries
    assert td * 5 < deg * 2


def test_workload_order_suffix():
    g, r, _ = P.workload("grid24@td")
    assert np.array_equal(r, P.hybrid_rank(g, None))
    g, r, _ = P.workload("ba2000@hybrid5")
    assert np.array_equal(r, P.hybrid_rank(g, 5))
    with pytest.raises(KeyError):
        P.workload("grid24@bogus")
