"""Landmark filter of pruning rule 2 (Section "Landmark-Based Filtering").

The landmark distances the build computes are checked against breadth-first
search in the oracle (exact, 16 bits), and the index built with the
filter, at several landmark counts and with it off, is checked against the
oracle bit for bit: the filter may only change speed."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import pspc_inputs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pspc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_00977_gb300 as lib

    lib.load()
    return lib


def _order(rank):
    order = np.empty(len(rank), np.int64)
    order[rank] = np.arange(len(rank))
    return order


def expected_landmarks(g, rank, k):
    """dist[v, j] = sd(v, j-th highest-ranked vertex) from oracle BFS;
    0xFFFF when unreachable or when the graph has no j-th vertex."""
    out = np.full((g.n, k), 0xFFFF, np.uint16)
    order = _order(rank)
    for j in range(min(k, g.n)):
        d, _, _ = oracle.bfs_count(g, int(order[j]))
        ok = d >= 0
        out[ok, j] = d[ok]
    return out


def path_graph(n):
    e = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1)
    return P.csr_from_edges(n, e, f"path{n}")


GRAPHS = {
    "ba2000": lambda: P.workload("ba2000")[:2],
    "rmat12_ef16": lambda: P.workload("rmat12_ef16")[:2],
    "grid64": lambda: P.workload("grid64")[:2],
    "path300": lambda: (lambda g: (g, P.degree_rank(g, "random", 5)))(path_graph(300)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("k", [1, 17, 32, 64])
def test_landmark_distances_equal_bfs(pspc, name, k):
    g, rank = GRAPHS[name]()
    ix = pspc.Index.from_graph(g, rank, landmarks=k)
    try:
        assert ix.stats()["landmarks"] == k
        got = ix.landmarks()
        assert got.shape == (g.n, k)
        assert np.array_equal(got, expected_landmarks(g, rank, k))
    finally:
        ix.free()


def test_landmarks_off(pspc):
    g, rank = GRAPHS["ba2000"]()
    ix = pspc.Index.from_graph(g, rank, landmarks=-1)
    try:
        assert ix.stats()["landmarks"] == 0
        assert ix.landmarks().shape == (g.n, 0)
        assert all(l["landmark_pruned"] == 0 for l in ix.level_stats())
    finally:
        ix.free()


def test_batch_landmarks_per_graph(pspc):
    graphs = [(n, rp, col, rk) for n, rp, col, rk in P.ba_batch(count=5, n_range=(20, 400), m_range=(1, 3), seed=77)]
    tiny = path_graph(5)
    graphs.append((tiny.n, tiny.row_ptr, tiny.col, P.degree_rank(tiny, "id")))
    k = 32
    ix = pspc.Index.build_batch(graphs, landmarks=k)
    try:
        got = ix.landmarks()
        base = 0
        for n, rp, col, rk in graphs:
            g = P.Graph(n, rp, col)
            assert np.array_equal(got[base:base + n], expected_landmarks(g, rk, k)), base
            base += n
        assert base == got.shape[0]
    finally:
        ix.free()


@pytest.mark.parametrize("name", ["ba2000", "rmat12_ef16", "grid64"])
@pytest.mark.parametrize("k", [-1, 1, 17, 64])
def test_index_independent_of_landmarks(pspc, name, k):
    g, rank = GRAPHS[name]()
    ref = oracle.OracleIndex(g, rank).export()
    ix = pspc.Index.from_graph(g, rank, landmarks=k)
    try:
        off, hub, dist, cnt, ovf = ix.export()
        assert np.array_equal(off, ref.off) and np.array_equal(hub, ref.hub)
        assert np.array_equal(dist, ref.dist) and np.array_equal(cnt, ref.cnt) and np.array_equal(ovf, ref.ovf)
        dropped = sum(l["landmark_pruned"] for l in ix.level_stats())
        if k > 0 and name != "grid64":
            assert dropped > 0
    finally:
        ix.free()


def test_landmark_option_range(pspc):
    g, rank = GRAPHS["ba2000"]()
    for bad in (-2, 65):
        with pytest.raises(pspc.PSPCError) as e:
            pspc.Index.from_graph(g, rank, landmarks=bad)
        assert e.value.code == 1
