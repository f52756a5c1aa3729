"""Pins for the CPU oracle (no GPU): the paper's worked example, closed
forms, exact big-integer brute force, invariants and the overflow rule."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from tests import _graphs as G
from pspc_inputs import Graph, csr_from_edges

M64 = 1 << 64


def c_labels(g, rank):
    ix = oracle.OracleIndex(g, rank)
    return ix, ix.export()


def assert_matches_exact(lab, exact_labels):
    """Oracle labels (mod 2^64 + flag) equal exact big-int labels."""
    for v, ent in enumerate(exact_labels):
        got = lab.of(v)
        assert [(h, d) for h, d, _, _ in got] == [(h, d) for h, d, _ in ent], v
        for (h, d, c, f), (_, _, ce) in zip(got, ent):
            assert c == ce % M64, (v, h)
            assert f == int(ce >= M64), (v, h)


# --- the paper's example (Table "Shortest Path Counting Labels of Fig. 1") ---

def test_paper_table_c_oracle():
    g, rank, table, _ = G.load_paper_table()
    ix, lab = c_labels(g, rank)
    assert ix.entries == 35
    for v in range(10):
        assert [(h, d, c) for h, d, c, _ in lab.of(v)] == table[v], v


def test_paper_table_brute():
    g, rank, table, _ = G.load_paper_table()
    L = brute.labels(g.n, g.edges(), rank)
    assert sum(map(len, L)) == 35
    for v in range(10):
        assert L[v] == table[v]


def test_paper_worked_query():
    g, rank, _, (s, t, d, c) = G.load_paper_table()
    assert (d, c) == (3, 4)
    ix = oracle.OracleIndex(g, rank)
    qd, qc, qf, _ = ix.query(np.array([[s, t], [t, s]]))
    assert qd.tolist() == [d, d] and qc.tolist() == [c, c] and qf.tolist() == [0, 0]
    assert brute.spc(g.n, g.edges(), s, t) == (d, c)


def test_paper_table_all_queries_equal_bfs():
    g, rank, _, _ = G.load_paper_table()
    ix = oracle.OracleIndex(g, rank)
    pairs = np.array(list(itertools.product(range(10), range(10))), np.int32)
    qd, qc, qf, _ = ix.query(pairs)
    allp = brute.spc_all(g.n, g.edges())
    for k, (s, t) in enumerate(pairs):
        d, c = allp[s]
        assert qd[k] == d[t] and qc[k] == c[t]


# --- brute force itself against textbook counts ---

@pytest.mark.parametrize("case", range(len(G.closed_forms())))
def test_brute_bfs_closed_forms(case):
    g, s, t, sd, cnt = G.closed_forms()[case]
    assert brute.spc(g.n, g.edges(), s, t) == (sd, cnt)


# --- C oracle against brute force ---

def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


def test_exhaustive_5_vertices_all_ranks_sampled():
    rng = np.random.default_rng(5)
    n = 5
    for edges in _all_graphs(n):
        g = csr_from_edges(n, np.array(edges, dtype=np.int64).reshape(-1, 2))
        for _ in range(2):
            rank = rng.permutation(n).astype(np.int32)
            _, lab = c_labels(g, rank)
            assert_matches_exact(lab, brute.labels(n, edges, rank))


def test_exhaustive_4_vertices_every_rank():
    n = 4
    for edges in _all_graphs(n):
        g = csr_from_edges(n, np.array(edges, dtype=np.int64).reshape(-1, 2))
        for perm in itertools.permutations(range(n)):
            rank = np.array(perm, np.int32)
            _, lab = c_labels(g, rank)
            assert_matches_exact(lab, brute.labels(n, edges, rank))


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_vs_brute(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 40))
    p = float(rng.choice([0.08, 0.15, 0.3]))
    g = G.gnp(n, p, seed)
    rank = G.random_rank(n, seed) if seed % 2 else G.degree_rank(g)
    _, lab = c_labels(g, rank)
    assert_matches_exact(lab, brute.labels(n, g.edges(), rank))


@pytest.mark.parametrize("k", [3, 4])
def test_hypercube_and_grid_labels_vs_brute(k):
    for g in (G.hypercube(k), G.grid(k + 1)):
        for rank in (G.degree_rank(g), G.random_rank(g.n, k)):
            _, lab = c_labels(g, rank)
            assert_matches_exact(lab, brute.labels(g.n, g.edges(), rank))


# --- ESPC: the query answers every pair exactly ---

@pytest.mark.parametrize("case", range(len(G.closed_forms())))
def test_query_closed_forms(case):
    g, s, t, sd, cnt = G.closed_forms()[case]
    for rank in (G.degree_rank(g), G.random_rank(g.n, case)):
        ix = oracle.OracleIndex(g, rank)
        qd, qc, qf, _ = ix.query(np.array([[s, t], [t, s], [s, s]]))
        assert qd.tolist() == [sd, sd, 0]
        assert qc.tolist() == [cnt % M64, cnt % M64, 1]
        assert qf.tolist() == [int(cnt >= M64)] * 2 + [0]


@pytest.mark.parametrize("seed", range(6))
def test_query_all_pairs_vs_exact_bfs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(10, 60))
    g = G.gnp(n, float(rng.choice([0.05, 0.1, 0.2])), 50 + seed)
    rank = G.random_rank(n, seed)
    ix = oracle.OracleIndex(g, rank)
    pairs = np.array(list(itertools.product(range(n), range(n))), np.int32)
    qd, qc, qf, _ = ix.query(pairs)
    allp = brute.spc_all(n, g.edges())
    for k, (s, t) in enumerate(pairs):
        d, c = allp[s]
        if t in d:
            assert (qd[k], qc[k], qf[k]) == (d[t], c[t] % M64, int(c[t] >= M64))
        else:
            assert (qd[k], qc[k], qf[k]) == (oracle.UNREACHED, 0, 0)


def test_query_ba2000_all_pairs_vs_bfs():
    """Workload ba2000 (n=2,000): all 4,000,000 ordered pairs against
    breadth-first counting from every source."""
    import pspc_inputs as P

    g, rank, _ = P.workload("ba2000")
    ix = oracle.OracleIndex(g, rank)
    n = g.n
    s = np.repeat(np.arange(n, dtype=np.int32), n)
    t = np.tile(np.arange(n, dtype=np.int32), n)
    qd, qc, qf, _ = ix.query(np.stack([s, t], 1))
    qd = qd.reshape(n, n)
    qc = qc.reshape(n, n)
    for src in range(n):
        d, c, f = oracle.bfs_count(g, src)
        assert np.array_equal(qd[src].astype(np.int32), np.where(d < 0, 0xFFFF, d))
        assert np.array_equal(qc[src], c)
    assert not qf.any()


# --- overflow rule: values mod 2^64, flag iff exact >= 2^64 ---

@pytest.mark.parametrize("k", [63, 64, 65])
def test_diamond_chain_label_overflow(k):
    g = G.diamond_chain(k)
    rank = np.arange(g.n, dtype=np.int32)  # a_0 highest: its column has 2^k at a_k
    _, lab = c_labels(g, rank)
    ent = [e for e in lab.of(3 * k) if e[0] == 0]
    assert ent == [(0, 2 * k, (1 << k) % M64, int(k >= 64))]


def test_grid_counts_overflow_vs_bigint():
    g = G.grid(36)  # corner-to-corner C(70,35) > 2^64
    rank = G.random_rank(g.n, 7)
    ix = oracle.OracleIndex(g, rank)
    pairs = np.array([[0, g.n - 1], [5, g.n - 40], [g.n - 1, 0]], np.int32)
    qd, qc, qf, _ = ix.query(pairs)
    for k, (s, t) in enumerate(pairs):
        d, c = brute.spc(g.n, g.edges(), int(s), int(t))
        assert (qd[k], qc[k], qf[k]) == (d, c % M64, int(c >= M64))
    assert qf[0] == 1


# --- structure and invariants ---

def test_trees_have_unit_counts():
    for seed in range(4):
        g = G.random_tree(80, seed)
        ix = oracle.OracleIndex(g, G.random_rank(g.n, seed))
        lab = ix.export()
        assert (lab.cnt == 1).all()


def test_isolated_vertices_and_components():
    g = csr_from_edges(7, np.array([(0, 1), (1, 2), (4, 5)]))
    rank = np.array([3, 0, 4, 6, 1, 5, 2], np.int32)
    ix = oracle.OracleIndex(g, rank)
    lab = ix.export()
    assert lab.of(3) == [(3, 0, 1, 0)] and lab.of(6) == [(6, 0, 1, 0)]
    qd, qc, qf, _ = ix.query(np.array([[0, 4], [3, 3], [3, 6], [0, 2]]))
    assert qd.tolist() == [0xFFFF, 0, 0xFFFF, 2]
    assert qc.tolist() == [0, 1, 0, 1]


def test_labels_invariant_under_vertex_renaming():
    """The index is a function of (G, order): renaming vertex ids and
    carrying the order along renames the labels and changes nothing else."""
    import pspc_inputs as P

    g = P.barabasi_albert(300, 3, 9)
    rank = G.degree_rank(g)
    perm = np.random.default_rng(4).permutation(g.n)  # new id of old vertex
    e = g.edges()
    g2 = csr_from_edges(g.n, perm[e])
    rank2 = np.empty(g.n, np.int32)
    rank2[perm] = rank
    lab = oracle.OracleIndex(g, rank).export()
    lab2 = oracle.OracleIndex(g2, rank2).export()
    for v in range(g.n):
        a = [(perm[h], d, c, f) for h, d, c, f in lab.of(v)]
        assert a == lab2.of(int(perm[v]))


def test_hub_prefix_build_is_restriction_of_full_index():
    import pspc_inputs as P

    g = P.barabasi_albert(400, 3, 2)
    rank = G.degree_rank(g)
    full = oracle.OracleIndex(g, rank).export()
    part_ix = oracle.OracleIndex(g, rank, max_hubs=37)
    part = part_ix.export()
    assert part_ix.hubs_done == 37
    for v in range(g.n):
        keep = [e for e in full.of(v) if rank[e[0]] < 37]
        assert part.of(v) == keep


def test_hub_column_checker_matches_index():
    import pspc_inputs as P

    g = P.barabasi_albert(500, 4, 3)
    rank = G.random_rank(g.n, 1)
    lab = oracle.OracleIndex(g, rank).export()
    col = {}
    for v in range(g.n):
        for h, d, c, f in lab.of(v):
            col[(h, v)] = (d, c, f)
    for w in [0, 17, 123, 499, int(np.argmin(rank)), int(np.argmax(rank))]:
        d, c, f = oracle.hub_column(g, rank, w)
        for v in range(g.n):
            if d[v] == oracle.UNREACHED:
                assert (w, v) not in col
            else:
                assert col[(w, v)] == (d[v], c[v], f[v])


def test_labels_sorted_by_hub_rank_and_self_entry_last():
    import pspc_inputs as P

    g = P.barabasi_albert(300, 2, 5)
    rank = G.random_rank(g.n, 3)
    lab = oracle.OracleIndex(g, rank).export()
    for v in range(g.n):
        ent = lab.of(v)
        r = [rank[h] for h, _, _, _ in ent]
        assert r == sorted(r) and len(set(r)) == len(r)
        assert ent[-1][:3] == (v, 0, 1)
        assert all(rank[h] <= rank[v] for h, _, _, _ in ent)


def test_rank_must_be_permutation():
    g = G.path(4)
    with pytest.raises(ValueError):
        oracle.OracleIndex(g, np.array([0, 1, 1, 2], np.int32))


def test_ba_batch_is_seeded_and_pool_independent():
    import pspc_inputs as P

    a = P.ba_batch(6, n_range=(50, 300), m_range=(1, 5), seed=4)
    b = P.ba_batch(6, n_range=(50, 300), m_range=(1, 5), seed=4, workers=2)
    assert len(a) == 6
    for x, y in zip(a, b):
        assert x[0] == y[0] and all(np.array_equal(u, v) for u, v in zip(x[1:], y[1:]))


# --- the parallel pair counter and the whole-index column checker ---

def test_spc_pairs_vs_exact_bfs_and_closed_forms():
    """oracle.spc_pairs (breadth-first counting per source, in parallel)
    equals exact big-integer counting on random graphs, every pair, and the
    textbook counts, overflow flags included."""
    for seed in range(4):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(10, 50))
        g = G.gnp(n, 0.12, 70 + seed)
        pairs = np.array(list(itertools.product(range(n), range(n))), np.int32)
        allp = brute.spc_all(n, g.edges())
        perm = rng.permutation(len(pairs))
        qd, qc, qf, th = oracle.spc_pairs(g, pairs[perm])
        assert th >= 1
        for k, (s, t) in enumerate(pairs[perm]):
            d, c = allp[s]
            if t in d:
                assert (qd[k], qc[k], qf[k]) == (d[t], c[t] % M64, int(c[t] >= M64))
            else:
                assert (qd[k], qc[k], qf[k]) == (oracle.UNREACHED, 0, 0)
    for g, s, t, sd, cnt in G.closed_forms():
        qd, qc, qf, _ = oracle.spc_pairs(g, np.array([[s, t], [t, s], [s, s]], np.int32))
        assert qd.tolist() == [sd, sd, 0]
        assert qc.tolist() == [cnt % M64, cnt % M64, 1]
        assert qf.tolist() == [int(cnt >= M64)] * 2 + [0]


def _brute_export(n, edges, rank):
    """Exact labels from the definition, in the export layout (counts mod
    2^64 and flags)."""
    L = brute.labels(n, edges, rank)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in L])
    flat = [e for x in L for e in x]
    hub = np.array([h for h, _, _ in flat], np.int32)
    dist = np.array([d for _, d, _ in flat], np.uint16)
    cnt = np.array([c % M64 for _, _, c in flat], np.uint64)
    ovf = np.array([int(c >= M64) for _, _, c in flat], np.uint8)
    return off, hub, dist, cnt, ovf


def test_check_columns_accepts_the_definition_and_finds_planted_mistakes():
    """oracle.check_columns passes the exact labels of the definition on
    graphs with several components and overflowing counts, and reports a
    mistake planted anywhere: a changed distance, count or flag, a dropped
    entry, an extra entry (caught by the entry total) and a swapped hub."""
    cases = [(G.gnp(40, 0.1, 3), 5), (G.grid(36), 7), (G.diamond_chain(65), 2)]
    for g, seed in cases:
        rank = G.random_rank(g.n, seed)
        exp = _brute_export(g.n, g.edges(), rank)
        bad, ent, _ = oracle.check_columns(g, rank, np.arange(g.n), *exp)
        assert bad == 0 and ent == int(exp[0][-1])
        rng = np.random.default_rng(seed)
        E = int(exp[0][-1])
        i = int(rng.integers(0, E))
        for field, delta in ((2, 1), (3, 1), (4, 1)):
            m = [a.copy() for a in exp]
            m[field][i] = m[field][i] + delta if field != 4 else 1 - m[field][i]
            bad, _, first = oracle.check_columns(g, rank, np.arange(g.n), *m)
            assert bad >= 1 and first[0][0] == exp[1][i]
        # drop the entry i: its vertex loses one entry
        v = int(np.searchsorted(exp[0], i, side="right") - 1)
        keep = np.ones(E, bool)
        keep[i] = False
        off2 = exp[0].copy()
        off2[v + 1:] -= 1
        dropped = (off2, exp[1][keep], exp[2][keep], exp[3][keep], exp[4][keep])
        bad, ent, _ = oracle.check_columns(g, rank, np.arange(g.n), *dropped)
        assert bad == 1 and ent == E
        # a hub swapped for another vertex's id: its own entry goes missing
        m = [a.copy() for a in exp]
        j = int(np.flatnonzero(m[2] > 0)[0])  # not a self entry
        m[1][j] = int(np.argmax(rank))  # the lowest-ranked vertex is nobody's hub but its own
        bad, _, _ = oracle.check_columns(g, rank, np.arange(g.n), *m)
        assert bad >= 1
        # an extra entry: every expected entry is still found, and the total
        # the definition gives is below the index size
        v = int(np.argmin(rank))  # the highest-ranked vertex has only its self entry
        x = int(np.argsort(rank)[1])
        off3 = exp[0].copy()
        off3[v + 1:] += 1
        pos = int(exp[0][v]) + 1  # after v's self entry: ranks stay increasing
        extra = (off3, np.insert(exp[1], pos, x), np.insert(exp[2], pos, 1), np.insert(exp[3], pos, 1),
                 np.insert(exp[4], pos, 0))
        bad, ent, _ = oracle.check_columns(g, rank, np.arange(g.n), *extra)
        assert bad == 0 and ent == E and int(off3[-1]) == E + 1


def test_hub_columns_equal_the_definition():
    """oracle.hub_columns (many hub columns, in parallel) equals the exact
    labels of the definition, hub by hub, overflow flags included."""
    for g, seed in ((G.gnp(50, 0.08, 9), 1), (G.grid(36), 4)):
        rank = G.random_rank(g.n, seed)
        L = brute.labels(g.n, g.edges(), rank)
        hubs = np.random.default_rng(seed).permutation(g.n)[:40]
        d, c, f = oracle.hub_columns(g, rank, hubs)
        for i, w in enumerate(hubs):
            for v in range(g.n):
                e = [(dd, cc) for h, dd, cc in L[v] if h == w]
                if e:
                    assert (d[i, v], c[i, v], f[i, v]) == (e[0][0], e[0][1] % M64, int(e[0][1] >= M64))
                else:
                    assert (d[i, v], c[i, v], f[i, v]) == (oracle.UNREACHED, 0, 0)
