"""Landmark filter of pruning rule 2 (Section "Landmark-Based Filtering").

The landmarks the build chooses are checked against their definition
(highest-ranked vertices, then spread ones chosen by the stated rule from
oracle BFS distances), their distances against breadth-first search in the
oracle (exact, 16 bits), and the index built with the filter, at several
landmark counts and with it off, against the oracle bit for bit: the filter
may only change speed."""
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


def expected_landmark_vertices(g, rank, k):
    """The landmarks of one graph by their definition: the min(k, 32)
    highest-ranked vertices; when k > 32 and n > 4k, then k - 32 spread
    vertices, each maximising the smaller of its distance to the first 32
    and its landmark lower bound to the spread ones before it (0 for a
    vertex no first landmark reaches; 0xFFFF when exactly one of the two is
    reached by some first landmark), ties to the higher rank; none when no
    vertex is 8 or more from the first 32. Distances from oracle BFS."""
    order = _order(rank)
    k1 = k if (k <= 32 or g.n <= 4 * k) else 32
    ids = [int(order[j]) for j in range(min(k1, g.n))]
    if k1 < k:
        D = np.stack([oracle.bfs_count(g, v)[0] for v in ids]).astype(np.int64)
        if 2 * D.max() < 16:  # labels stop short of the levels that test spread landmarks
            return ids + [-1] * (k - len(ids))
        R = D >= 0
        score = np.where(R.any(axis=0), np.where(R, D, 1 << 40).min(axis=0), 0)
        for _ in range(k - k1):
            top = np.nonzero(score == score.max())[0]
            p = int(top[np.argmin(rank[top])])
            ids.append(p)
            one = (R ^ R[:, p:p + 1]).any(axis=0)
            diff = np.where(R & R[:, p:p + 1], np.abs(D - D[:, p:p + 1]), 0).max(axis=0)
            score = np.minimum(score, np.where(one, 0xFFFF, diff))
    return ids + [-1] * (k - len(ids))


def expected_landmarks(g, rank, k, ids=None):
    """dist[v, j] = sd(v, landmark j) from oracle BFS; 0xFFFF when
    unreachable or when the graph has no landmark j. Landmarks: ids, else
    the k highest-ranked vertices."""
    out = np.full((g.n, k), 0xFFFF, np.uint16)
    if ids is None:
        order = _order(rank)
        ids = [int(order[j]) for j in range(min(k, g.n))]
    for j, v in enumerate(ids):
        if v < 0:
            continue
        d, _, _ = oracle.bfs_count(g, int(v))
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
@pytest.mark.parametrize("k", [1, 17, 32, 64, 100, 128])
def test_landmark_distances_equal_bfs(pspc, name, k):
    g, rank = GRAPHS[name]()
    ix = pspc.Index.from_graph(g, rank, landmarks=k)
    try:
        assert ix.stats()["landmarks"] == k
        ids = expected_landmark_vertices(g, rank, k)
        assert ix.landmark_vertices().tolist() == ids
        got = ix.landmarks()
        assert got.shape == (g.n, k)
        assert np.array_equal(got, expected_landmarks(g, rank, k, ids))
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


def test_spread_landmarks_lie_far_apart(pspc):
    """On a grid the spread landmarks (33..64) are 32 distinct vertices,
    none of them a highest-ranked one, the first at a largest distance from
    landmarks 1..32; a batch index has no landmark vertex list."""
    g, rank = GRAPHS["grid64"]()
    ix = pspc.Index.from_graph(g, rank, landmarks=64)
    try:
        ids = ix.landmark_vertices()
        D = ix.landmarks()
        first = D[:, :32].astype(np.int64)
        reach = (first != 0xFFFF).any(axis=1)
        score = np.where(first == 0xFFFF, 1 << 40, first).min(axis=1)
        assert score[ids[32]] == score[reach].max()
        assert len(set(ids[32:].tolist())) == 32 and not set(ids[32:].tolist()) & set(ids[:32].tolist())
        assert (D[ids[32:]][:, 32:][~np.eye(32, dtype=bool)] > 0).all()
        with pytest.raises(pspc.PSPCError):
            graphs = [(n, rp, col, rk) for n, rp, col, rk in P.ba_batch(count=2, n_range=(300, 400), m_range=(1, 3), seed=5)]
            bix = pspc.Index.build_batch(graphs, landmarks=64)
            try:
                bix.landmark_vertices()
            finally:
                bix.free()
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
@pytest.mark.parametrize("k", [-1, 1, 17, 64, 128])
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
    graphs = [(n, rp, col, rk) for n, rp, col, rk in P.ba_batch(count=3, n_range=(20, 40), m_range=(1, 2), seed=3)]
    with pytest.raises(pspc.PSPCError) as e:
        pspc.Index.build_batch(graphs, landmarks=65)
    assert e.value.code == 1
    for bad in (-2, 129):
        with pytest.raises(pspc.PSPCError) as e:
            pspc.Index.from_graph(g, rank, landmarks=bad)
        assert e.value.code == 1
